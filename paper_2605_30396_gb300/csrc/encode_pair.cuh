// Batch-OMP with two tiles in flight per CTA (Sec. 2.1: OMP against the
// dictionary, one greedy atom at a time, least-squares re-fit), for s <= 8.
//
// Included by encode.cu inside namespace dlsh::enc (it uses that file's
// operand packing, key networks and constants).
//
// Each CTA runs two groups of eight warps; group g owns its own tiles of 128
// signals (tiles blockIdx.x + (2k + g) * gridDim.x).  While one group solves
// (Cholesky update, least squares and residual, which wait on L2 loads), the
// tensor pipe runs the other group's correlations and that group selects.
//   warp 17  TMA producer: streams 64-atom chunks of the packed dictionary
//            through a ring, in the order the MMA warp consumes them.
//   warp 16  MMA issuer: serves the groups' OMP iterations alternately
//            (group 0 iteration it, group 1 iteration it, ...).  FP32: the
//            group's residual, staged in shared memory as TF32 hi/lo parts,
//            is first copied into the group's tensor-memory A columns
//            (tcgen05.cp), and the 3xTF32 MMAs read A from tensor memory;
//            BF16/FP8: A stays in shared memory (one region per group).
//   warps 0-15  two groups of eight.  Selection: thread (lane, warp w of the
//            group) reads TMEM lane 32 (w % 4) + lane, i.e. one row, over the
//            column half w / 4 of every chunk.  Solver: two sub-lanes per
//            signal, each owning 24 of the 48 padded dimensions.
// Tensor memory: 256 columns per group.  FP32: A hi at columns 0..47, A lo at
// 48..95, two 64-column accumulator buffers at 128..255.  BF16/FP8: four
// 64-column accumulator buffers.

constexpr int PBN = 64;   // atoms per chunk
constexpr int PQC = 32;   // chunk columns read by one selection thread
constexpr int PGT = 256;  // threads per group

struct PairPlan {
  int prec, top4, ib, K, Kp, nchunks, stages, s;
  uint32_t chunk_bytes, a_bytes;
  uint32_t off_a[2], off_L[2], off_sel[2], off_y[2], off_g[2], off_idg[2], off_cand[2], off_r[2];
  uint32_t off_sig, off_ring, off_bar, smem;
};

struct PairArgs {
  const float* X;
  int64_t N;
  const float* D32p;
  const float* G;
  const uint8_t* img;
  const float* sigma;
  uint16_t* idx;
  float* coef;
  uint8_t* nnz;
  float* resid_sq;
  float eps;
  uint32_t* status;
  long long budget;
  const long long* n_dev;  // optional: signal count read on the device (overrides N)
  PairPlan p;
};

inline int make_pair_plan(int K, int s, int code, PairPlan& p, int smem_limit = SMEM_LIMIT) {
  if (s > 8) return DLSH_ERR_UNSUPPORTED;
  const int prec = operand_precision(code, &p.top4);
  p.prec = prec;
  p.K = K;
  p.s = s;
  p.nchunks = (K + PBN - 1) / PBN;
  p.Kp = p.nchunks * PBN;
  p.ib = 5;
  while ((1 << (p.ib - 5)) < p.nchunks) ++p.ib;
  p.a_bytes = TILE_M * op_kb(prec) * 16 * op_parts(prec);
  p.chunk_bytes = PBN * op_kb(prec) * 16 * op_parts(prec);
  uint32_t off = 0;
  auto take = [&](uint32_t bytes) {
    uint32_t o = (off + 1023u) & ~1023u;
    off = o + bytes;
    return o;
  };
  // FP32: one staging area shared by the groups (A itself lives in TMEM)
  p.off_a[0] = take(p.a_bytes);
  p.off_a[1] = prec == 0 ? p.off_a[0] : take(p.a_bytes);
  for (int g = 0; g < 2; ++g) {
    p.off_L[g] = take(36 * TILE_M * 4);
    p.off_sel[g] = take(8 * TILE_M * 4);
    p.off_y[g] = take(8 * TILE_M * 4);
    p.off_g[g] = take(8 * TILE_M * 4);
    p.off_idg[g] = take(8 * TILE_M * 4);
    p.off_cand[g] = take(p.top4 ? TILE_M * 2 * 4 * 4 : TILE_M * 2 * 8);
    p.off_r[g] = take(prec == 0 ? 0 : PGT * 24 * 4);
  }
  p.off_sig = take(prec == 2 ? p.Kp * 4 : 0);
  p.off_bar = take(1024);
  const uint32_t fixed = (off + 1023u) & ~1023u;
  if (fixed >= static_cast<uint32_t>(smem_limit)) return DLSH_ERR_UNSUPPORTED;
  int fit = static_cast<int>((smem_limit - fixed) / p.chunk_bytes);
  if (fit > 32) fit = 32;
  if (fit < 3) return DLSH_ERR_UNSUPPORTED;
  p.stages = fit;
  p.off_ring = fixed;
  p.smem = fixed + p.stages * p.chunk_bytes;
  return DLSH_OK;
}

// Butterfly over the two sub-lanes of one signal (lanes 2k, 2k+1).
__device__ __forceinline__ unsigned pair_mask() { return 0x3u << ((threadIdx.x & 31) & ~1u); }
__device__ __forceinline__ float pair_sum(float v) { return v + __shfl_xor_sync(pair_mask(), v, 1); }
__device__ __forceinline__ float pair_max(float v) {
  return fmaxf(v, __shfl_xor_sync(pair_mask(), v, 1));
}

// Sub-lane u's 24 dims of row `row` into the A operand (FP8 scaled by inv_rho).
template <int PREC>
__device__ __forceinline__ void write_a_part24(uint8_t* A, int row, int u, const float (&r)[24],
                                               float inv_rho) {
  constexpr uint32_t LBO = TILE_M * 16;
  if constexpr (PREC == 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 pk;
      pk.x = pack_bf16x2(r[8 * k + 0], r[8 * k + 1]);
      pk.y = pack_bf16x2(r[8 * k + 2], r[8 * k + 3]);
      pk.z = pack_bf16x2(r[8 * k + 4], r[8 * k + 5]);
      pk.w = pack_bf16x2(r[8 * k + 6], r[8 * k + 7]);
      *reinterpret_cast<uint4*>(A + (3 * u + k) * LBO + row * 16) = pk;
    }
  } else if constexpr (PREC == 0) {
    constexpr uint32_t PART = TILE_M * 12 * 16;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int kb = 6 * u + k;
      float4 hi, lo;
      hi.x = to_tf32(r[4 * k + 0]);
      hi.y = to_tf32(r[4 * k + 1]);
      hi.z = to_tf32(r[4 * k + 2]);
      hi.w = to_tf32(r[4 * k + 3]);
      lo.x = to_tf32(r[4 * k + 0] - hi.x);
      lo.y = to_tf32(r[4 * k + 1] - hi.y);
      lo.z = to_tf32(r[4 * k + 2] - hi.z);
      lo.w = to_tf32(r[4 * k + 3] - hi.w);
      *reinterpret_cast<float4*>(A + kb * LBO + row * 16) = hi;
      *reinterpret_cast<float4*>(A + PART + kb * LBO + row * 16) = lo;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int e = 24 * u + 4 * k;
      const uint32_t w = pack_e4m3x4(r[4 * k] * inv_rho, r[4 * k + 1] * inv_rho,
                                     r[4 * k + 2] * inv_rho, r[4 * k + 3] * inv_rho);
      *reinterpret_cast<uint32_t*>(A + (e >> 4) * LBO + row * 16 + (e & 15)) = w;
    }
  }
}

// One chunk of MMAs for the pair kernel: D[tmem] = A . B^T over K = 48 (64 for
// FP8), N = 64.  FP32: A (hi, lo) from tensor memory at a_tmem; else A from
// shared memory at a_addr.
template <int PREC>
__device__ __forceinline__ void issue_pair_chunk(uint32_t tmem_d, uint32_t a_tmem, uint32_t a_addr,
                                                 uint32_t b_addr) {
  if constexpr (PREC == 0) {
    constexpr uint32_t idesc = umma_idesc(2, 2, TILE_M, PBN);
    constexpr uint32_t B_LBO = PBN * 16, SBO = 128, B_PART = PBN * 12 * 16;
#pragma unroll
    for (int pass = 0; pass < 3; ++pass) {
      const uint32_t ao = pass == 2 ? 48u : 0u;    // lo(r) . hi(D)
      const uint32_t bo = pass == 1 ? B_PART : 0u;  // hi(r) . lo(D)
#pragma unroll
      for (int ks = 0; ks < 6; ++ks) {
        const uint64_t bd = umma_smem_desc(b_addr + bo + ks * 2 * B_LBO, B_LBO, SBO);
        umma_tf32_tmem_a(tmem_d, a_tmem + ao + ks * 8, bd, idesc, (pass | ks) != 0);
      }
    }
  } else {
    issue_chunk<PREC, PBN>(tmem_d, a_addr, b_addr);
  }
}

template <int PREC, bool T4>
__global__ void __launch_bounds__(NTHREADS, 1) encode_pair_kernel(const __grid_constant__ PairArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int SMAX = 8;
  constexpr int NBUF = PREC == 0 ? 2 : 4;
  constexpr uint32_t BUF0 = PREC == 0 ? 128u : 0u;
  const PairPlan& p = a.p;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long NS = a.n_dev ? *a.n_dev : a.N;
  const int ntiles = static_cast<int>((NS + TILE_M - 1) / TILE_M);
  const int Gd = static_cast<int>(gridDim.x), bidx = static_cast<int>(blockIdx.x);
  const int s = p.s;
  // rounds k in which group 0 / group 1 have a tile (tiles b + (2k + g) Gd)
  const int K0 = bidx < ntiles ? (ntiles - bidx + 2 * Gd - 1) / (2 * Gd) : 0;
  const int K1 = bidx + Gd < ntiles ? (ntiles - bidx - Gd + 2 * Gd - 1) / (2 * Gd) : 0;
  // position of job (g, k, it) in the MMA warp's order
  auto job_index = [&](int g, int k, int it) -> long long {
    return k < K1 ? 2LL * s * k + 2LL * it + g : 2LL * s * K1 + static_cast<long long>(s) * (k - K1) + it;
  };

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + p.off_bar);
  uint64_t* bar_a = bars;            // [2]
  uint64_t* bar_full = bars + 2;     // [2][4]
  uint64_t* bar_empty = bars + 10;   // [2][4]
  uint64_t* bar_stage = bars + 18;   // FP32: the staged A has been copied into TMEM
  uint64_t* bar_dfull = bars + 19;   // [stages]
  uint64_t* bar_dempty = bar_dfull + p.stages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_dempty + p.stages);
  volatile long long* stage_done = reinterpret_cast<volatile long long*>(smem + p.off_bar + 1000);

  if (tid == 0) {
    for (int g = 0; g < 2; ++g) {
      mbar_init(&bar_a[g], 1);
      for (int b = 0; b < NBUF; ++b) {
        mbar_init(&bar_full[g * 4 + b], 1);
        mbar_init(&bar_empty[g * 4 + b], 8);
      }
    }
    mbar_init(bar_stage, 1);
    for (int q = 0; q < p.stages; ++q) {
      mbar_init(&bar_dfull[q], 1);
      mbar_init(&bar_dempty[q], 1);
    }
    *stage_done = -1;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t ring_addr = smem_u32(smem + p.off_ring);

  if (warp == 17) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      long long ring = 0;
      bool ok = true;
      for (int k = 0; k < K0 && ok; ++k)
        for (int it = 0; it < s && ok; ++it)
          for (int g = 0; g < (k < K1 ? 2 : 1) && ok; ++g)
            for (int c = 0; c < p.nchunks; ++c, ++ring) {
              const int st = static_cast<int>(ring % p.stages);
              const uint32_t par = static_cast<uint32_t>((ring / p.stages) & 1) ^ 1u;
              if (!mbar_wait(&bar_dempty[st], par, a.budget)) {
                flag_status(a.status, ST_TIMEOUT);
                ok = false;
                break;
              }
              mbar_arrive_expect_tx(&bar_dfull[st], p.chunk_bytes);
              bulk_g2s(smem + p.off_ring + static_cast<size_t>(st) * p.chunk_bytes,
                       a.img + static_cast<size_t>(c) * p.chunk_bytes, p.chunk_bytes, &bar_dfull[st]);
            }
      // every slot's last fill has been consumed before the CTA exits
      for (long long f = ring > p.stages ? ring - p.stages : 0; ok && f < ring; ++f) {
        if (!mbar_wait(&bar_dempty[f % p.stages], static_cast<uint32_t>((f / p.stages) & 1), a.budget)) {
          flag_status(a.status, ST_TIMEOUT);
          ok = false;
        }
      }
    }
  } else if (warp == 16) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t aph[2] = {0u, 0u};
      long long cc[2] = {0, 0};
      long long ring = 0, job = 0;
      bool ok = true;
      for (int k = 0; k < K0 && ok; ++k)
        for (int it = 0; it < s && ok; ++it)
          for (int g = 0; g < (k < K1 ? 2 : 1) && ok; ++g, ++job) {
            if (!mbar_wait(&bar_a[g], aph[g], a.budget)) {
              flag_status(a.status, ST_TIMEOUT);
              ok = false;
              break;
            }
            aph[g] ^= 1u;
            tc_fence_after();
            const uint32_t tg = tmem_base + static_cast<uint32_t>(g) * 256u;
            if constexpr (PREC == 0) {
              // staged residual (TF32 hi, lo) -> this group's A columns; the
              // staging area is free again once the copies complete
              constexpr uint32_t LBO = TILE_M * 16, SBO = 128, PART = TILE_M * 12 * 16;
              const uint32_t sa = smem_u32(smem + p.off_a[0]);
#pragma unroll
              for (int part = 0; part < 2; ++part)
#pragma unroll
                for (int kk = 0; kk < 6; ++kk)
                  tmem_cp_128x256b(tg + part * 48 + kk * 8,
                                   umma_smem_desc(sa + part * PART + kk * 2 * LBO, LBO, SBO));
              tc_commit(bar_stage);
              if (!mbar_wait(bar_stage, static_cast<uint32_t>(job & 1), a.budget)) {
                flag_status(a.status, ST_TIMEOUT);
                ok = false;
                break;
              }
              *stage_done = job;
            }
            for (int c = 0; c < p.nchunks; ++c, ++ring, ++cc[g]) {
              const int st = static_cast<int>(ring % p.stages);
              const uint32_t dpar = static_cast<uint32_t>((ring / p.stages) & 1);
              const int buf = static_cast<int>(cc[g] % NBUF);
              const uint32_t epar = static_cast<uint32_t>((cc[g] / NBUF) & 1) ^ 1u;
              if (!mbar_wait(&bar_dfull[st], dpar, a.budget) ||
                  !mbar_wait(&bar_empty[g * 4 + buf], epar, a.budget)) {
                flag_status(a.status, ST_TIMEOUT);
                ok = false;
                break;
              }
              tc_fence_after();
              issue_pair_chunk<PREC>(tg + BUF0 + static_cast<uint32_t>(buf) * PBN, tg,
                                     smem_u32(smem + p.off_a[g]),
                                     ring_addr + static_cast<uint32_t>(st) * p.chunk_bytes);
              tc_commit(&bar_full[g * 4 + buf]);
              tc_commit(&bar_dempty[st]);
            }
          }
    }
  } else {
    // ------------------------------------------------ two groups: selection + solver
    const int g = warp >> 3, gw = warp & 7, gtid = tid - g * PGT;
    const uint32_t gbar = 1u + static_cast<uint32_t>(g);
    uint8_t* A = smem + p.off_a[g];
    float* Ls = reinterpret_cast<float*>(smem + p.off_L[g]);
    int* sel = reinterpret_cast<int*>(smem + p.off_sel[g]);
    float* ys = reinterpret_cast<float*>(smem + p.off_y[g]);
    float* gs = reinterpret_cast<float*>(smem + p.off_g[g]);
    float* idg = reinterpret_cast<float*>(smem + p.off_idg[g]);
    float* cv = reinterpret_cast<float*>(smem + p.off_cand[g]);       // [128][2]
    int* cj = reinterpret_cast<int*>(smem + p.off_cand[g] + TILE_M * 2 * 4);
    uint32_t* ckeys = reinterpret_cast<uint32_t*>(smem + p.off_cand[g]);  // T4: [128][2][4]
    float* rsm = reinterpret_cast<float*>(smem + p.off_r[g]);  // [24][256]
    float* sig = reinterpret_cast<float*>(smem + p.off_sig);
    if constexpr (PREC == 2) {
      for (int j = tid; j < p.Kp; j += 2 * PGT) sig[j] = a.sigma[j];
      // FP8 rows hold 64 bytes: bytes 48..63 are zero padding, written once
      for (int row = gtid; row < TILE_M; row += PGT)
        *reinterpret_cast<uint4*>(A + 3 * TILE_M * 16 + row * 16) = make_uint4(0, 0, 0, 0);
      named_bar_sync(3, 2 * PGT);
    }
    const int R1 = 32 * (gw & 3) + lane, h = gw >> 2;
    const int R2 = 16 * gw + (lane >> 1), u = lane & 1;
    const uint32_t trow = tmem_base + (static_cast<uint32_t>(32 * (gw & 3)) << 16) +
                          static_cast<uint32_t>(g) * 256u + BUF0 + static_cast<uint32_t>(h * PQC);
#define LS(rr, cc2) Ls[(((rr) * ((rr) + 1)) / 2 + (cc2)) * TILE_M + R2]
#define IDG(rr) idg[(rr) * TILE_M + R2]
    long long ccg = 0;
    bool ok = true;
    // FP32: the staging area may be written for job J once the copy of job
    // J - 1 into TMEM has completed (published by the MMA warp)
    auto wait_staging = [&](long long J) -> bool {
      if constexpr (PREC == 0) {
        const long long t0 = clock64();
        while (*stage_done < J - 1) {
          if (clock64() - t0 > a.budget) {
            flag_status(a.status, ST_TIMEOUT);
            return false;
          }
        }
      }
      return true;
    };
    const int ktiles = g == 0 ? K0 : K1;
    for (int k = 0; k < ktiles && ok; ++k) {
      const long long tile = static_cast<long long>(bidx) + (2LL * k + g) * Gd;
      const int K = p.K, nchunks = p.nchunks;
      const float eps2 = a.eps * a.eps;
      const int64_t g0 = tile * TILE_M;
      const int rows = static_cast<int>(NS - g0 < TILE_M ? NS - g0 : TILE_M);
      const bool in_tile = R2 < rows;
      const float* xr = a.X + (g0 + R2) * DLSH_D + 24 * u;
      auto load_x = [&](float (&x)[24]) {
#pragma unroll
        for (int q = 0; q < 24; ++q) x[q] = (in_tile && 24 * u + q < DLSH_D) ? __ldg(xr + q) : 0.f;
      };
      // -------- the signals are the first A operand
      float rn2;
      {
        float x[24];
        load_x(x);
        float part = 0.f;
#pragma unroll
        for (int q = 0; q < 24; ++q) part = fmaf(x[q], x[q], part);
        float inv = 1.f;
        if constexpr (PREC == 2) {
          float mx = 0.f;
#pragma unroll
          for (int q = 0; q < 24; ++q) mx = fmaxf(mx, fabsf(x[q]));
          mx = pair_max(mx);
          inv = mx > 0.f ? FP8_MAX / mx : 1.f;
        }
        if (wait_staging(job_index(g, k, 0)))
          write_a_part24<PREC>(A, R2, u, x, inv);
        else
          ok = false;
        if constexpr (PREC != 0) {
#pragma unroll
          for (int q = 0; q < 24; ++q) rsm[q * PGT + gtid] = x[q];
        }
        rn2 = pair_sum(part);
      }
      fence_proxy_async_smem();
      if (named_bar_or(gbar, PGT, !ok)) {
        ok = false;
        break;
      }
      if (gtid == 0) mbar_arrive(&bar_a[g]);
      const float xnorm = sqrtf(rn2);
      bool active = in_tile;
      int t = 0;

      for (int it = 0; it < s; ++it) {
        // ================= phase 1: selection over this thread's column half
        {
          uint32_t best = 0;
          int bestc = 0;
          const uint32_t vmask = 0x7fffffffu & ~((1u << p.ib) - 1u);
          uint32_t run[4] = {0u, 0u, 0u, 0u};
          for (int c = 0; c < nchunks; ++c, ++ccg) {
            const int buf = static_cast<int>(ccg % NBUF);
            if (!mbar_wait(&bar_full[g * 4 + buf], static_cast<uint32_t>((ccg / NBUF) & 1), a.budget)) {
              flag_status(a.status, ST_TIMEOUT);
              ok = false;
              break;
            }
            tc_fence_after();
            __syncwarp();
            uint32_t rr[PQC];
            tmem_ld32_issue(trow + static_cast<uint32_t>(buf * PBN), rr);
            tmem_ld32_wait(rr);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_empty[g * 4 + buf]);
            if constexpr (PREC == 2) {
              const int j0 = c * PBN + h * PQC;
#pragma unroll
              for (int q = 0; q < PQC; ++q) rr[q] = __float_as_uint(__uint_as_float(rr[q]) * sig[j0 + q]);
            }
            if constexpr (T4) {
#pragma unroll
              for (int q = 0; q < PQC; ++q) rr[q] = (rr[q] & vmask) | static_cast<uint32_t>(31 - q);
              uint32_t ct[4];
              top4_of8(rr, ct);
#pragma unroll
              for (int o = 8; o < PQC; o += 8) {
                uint32_t t8[4];
                top4_of8(rr + o, t8);
                merge_top4(ct, t8);
              }
              const uint32_t cf = ((1u << p.ib) - 32u) - static_cast<uint32_t>(c) * 32u;
#pragma unroll
              for (int i = 0; i < 4; ++i) ct[i] |= cf;
              merge_top4(run, ct);
            } else {
              uint32_t m0 = 0, m1 = 0;
#pragma unroll
              for (int q = 0; q < PQC; q += 2) {
                m0 = max(m0, (rr[q] & 0x7fffffe0u) | static_cast<uint32_t>(31 - q));
                m1 = max(m1, (rr[q + 1] & 0x7fffffe0u) | static_cast<uint32_t>(30 - q));
              }
              const uint32_t m = max(m0, m1);
              if ((m & ~31u) > (best & ~31u)) {
                best = m;
                bestc = c;
              }
            }
          }
          if constexpr (T4) {
#pragma unroll
            for (int i = 0; i < 4; ++i) ckeys[(R1 * 2 + h) * 4 + i] = run[i];
          } else {
            cv[R1 * 2 + h] = __uint_as_float(best & ~31u);
            cj[R1 * 2 + h] = bestc * PBN + h * PQC + 31 - static_cast<int>(best & 31u);
          }
        }
        if (named_bar_or(gbar, PGT, !ok)) {
          ok = false;
          break;
        }
        // ================= phase 2: merge, re-score, Cholesky, solve, residual
        if (active && rn2 <= eps2) active = false;
        if (active) {
          float r[24];
          int sl[SMAX];
#pragma unroll
          for (int m = 0; m < SMAX; ++m) sl[m] = m < t ? sel[m * TILE_M + R2] : 0;
          int js = -1;
          float best = -1.f;
          if constexpr (PREC == 0) {
#pragma unroll
            for (int qq = 0; qq < 2; ++qq) {
              const float v = cv[R2 * 2 + qq];
              const int j = cj[R2 * 2 + qq];
              if (j < K && (v > best || (v == best && j < js))) {
                best = v;
                js = j;
              }
            }
          } else {
#pragma unroll
            for (int q = 0; q < 24; ++q) r[q] = rsm[q * PGT + gtid];
            // candidates: T4, the row's exact low-precision top 4 (sub-lane u
            // reads half u's list, one butterfly round); else the winner of
            // each column half
            int cjr[4];
            if constexpr (T4) {
              const uint32_t imask = (1u << p.ib) - 1u;
              unsigned long long lst[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const uint32_t key = ckeys[(R2 * 2 + u) * 4 + i];
                const uint32_t col = imask - (key & imask);
                const uint32_t j = (col >> 5) * PBN + static_cast<uint32_t>(u * PQC) + (col & 31u);
                lst[i] = key == 0u ? 0ull
                                   : (static_cast<unsigned long long>(key & ~imask & 0x7fffffffu) << 32) |
                                         static_cast<unsigned long long>(0xFFFFFFFFu - j);
              }
              unsigned long long oth[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) oth[i] = __shfl_xor_sync(pair_mask(), lst[i], 1);
              merge_top4(lst, oth);
#pragma unroll
              for (int i = 0; i < 4; ++i)
                cjr[i] = lst[i] == 0ull ? 0x7fffffff
                                        : static_cast<int>(0xFFFFFFFFu - static_cast<uint32_t>(lst[i]));
            } else {
              cjr[0] = cj[R2 * 2 + 0];
              cjr[1] = cj[R2 * 2 + 1];
              cjr[2] = cjr[3] = 0x7fffffff;
            }
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const int j = cjr[qq];
              float c0 = 0.f;
              if (j < K) {
                const float4* dr = reinterpret_cast<const float4*>(a.D32p + static_cast<size_t>(j) * DPAD + 24 * u);
#pragma unroll
                for (int w4 = 0; w4 < 6; ++w4) {
                  const float4 dv = __ldg(dr + w4);
                  c0 = fmaf(r[4 * w4 + 0], dv.x, c0);
                  c0 = fmaf(r[4 * w4 + 1], dv.y, c0);
                  c0 = fmaf(r[4 * w4 + 2], dv.z, c0);
                  c0 = fmaf(r[4 * w4 + 3], dv.w, c0);
                }
              }
              c0 = fabsf(pair_sum(c0));
              if (j < K && (c0 > best || (c0 == best && j < js))) {
                best = c0;
                js = j;
              }
            }
          }
          {
            // an atom already in the support has the largest |c| only when every
            // correlation is at rounding level: the row stops
            bool dup = false;
#pragma unroll
            for (int m = 0; m < SMAX; ++m) dup |= (m < t && sl[m] == js);
            if (dup) js = -1;
          }
          if (js < 0 || !(best > CORR_STOP_REL * xnorm)) {
            active = false;
          } else {
            // the step for a support of t atoms, compiled once per t
            auto step = [&](auto tag) {
              constexpr int T = decltype(tag)::value;
              constexpr int TA = T > 0 ? T : 1;
              const float* Grow = a.G + static_cast<size_t>(js) * K;
              float gv[TA];
#pragma unroll
              for (int m = 0; m < T; ++m) gv[m] = __ldg(Grow + sl[m]);
              const float gjj = __ldg(Grow + js);
              float4 dj[6];
              {
                const float4* dr = reinterpret_cast<const float4*>(a.D32p + static_cast<size_t>(js) * DPAD + 24 * u);
#pragma unroll
                for (int w4 = 0; w4 < 6; ++w4) dj[w4] = __ldg(dr + w4);
              }
              load_x(r);  // r holds x until the residual is formed
              float w[TA];
              float wn2 = 0.f;
#pragma unroll
              for (int m = 0; m < T; ++m) {
                float acc = gv[m];
#pragma unroll
                for (int q = 0; q < m; ++q) acc = fmaf(-LS(m, q), w[q], acc);
                w[m] = acc * IDG(m);
                wn2 = fmaf(w[m], w[m], wn2);
              }
              const float ell2 = gjj - wn2;
              if (!(ell2 > PIVOT_MIN * gjj)) {
                active = false;
                return;
              }
              const float ell = sqrtf(ell2);
              const float iell = 1.f / ell;
#pragma unroll
              for (int m = 0; m < T; ++m) LS(T, m) = w[m];  // both sub-lanes store identical values
              LS(T, T) = ell;
              IDG(T) = iell;
              float bp = 0.f;
#pragma unroll
              for (int w4 = 0; w4 < 6; ++w4) {
                bp = fmaf(dj[w4].x, r[4 * w4 + 0], bp);
                bp = fmaf(dj[w4].y, r[4 * w4 + 1], bp);
                bp = fmaf(dj[w4].z, r[4 * w4 + 2], bp);
                bp = fmaf(dj[w4].w, r[4 * w4 + 3], bp);
              }
              float yv[TA];
#pragma unroll
              for (int m = 0; m < T; ++m) yv[m] = ys[m * TILE_M + R2];
              float yt = pair_sum(bp);
#pragma unroll
              for (int m = 0; m < T; ++m) yt = fmaf(-w[m], yv[m], yt);
              yt *= iell;
              ys[T * TILE_M + R2] = yt;
              sel[T * TILE_M + R2] = js;
              const float gt = yt * iell;
              float gam[TA];
#pragma unroll
              for (int m = T - 1; m >= 0; --m) {
                float acc = yv[m];
#pragma unroll
                for (int q = m + 1; q < T; ++q) acc = fmaf(-LS(q, m), gam[q], acc);
                acc = fmaf(-w[m], gt, acc);
                gam[m] = acc * IDG(m);
              }
#pragma unroll
              for (int m = 0; m < T; ++m) gs[m * TILE_M + R2] = gam[m];
              gs[T * TILE_M + R2] = gt;
              // residual r = x - D_I gamma on this sub-lane's 24 dims
              // the support atoms' rows in groups of up to 2, all loads of a
              // group issued before its FMAs (one L2 round trip per group)
#pragma unroll
              for (int m0 = 0; m0 < T; m0 += 2) {
                float4 dv[2][6];
#pragma unroll
                for (int mm = 0; mm < 2; ++mm)
                  if (m0 + mm < T) {
                    const float4* da =
                        reinterpret_cast<const float4*>(a.D32p + static_cast<size_t>(sl[m0 + mm]) * DPAD + 24 * u);
#pragma unroll
                    for (int w4 = 0; w4 < 6; ++w4) dv[mm][w4] = __ldg(da + w4);
                  }
#pragma unroll
                for (int mm = 0; mm < 2; ++mm)
                  if (m0 + mm < T) {
                    const float gm = gam[m0 + mm];
#pragma unroll
                    for (int w4 = 0; w4 < 6; ++w4) {
                      r[4 * w4 + 0] = fmaf(-gm, dv[mm][w4].x, r[4 * w4 + 0]);
                      r[4 * w4 + 1] = fmaf(-gm, dv[mm][w4].y, r[4 * w4 + 1]);
                      r[4 * w4 + 2] = fmaf(-gm, dv[mm][w4].z, r[4 * w4 + 2]);
                      r[4 * w4 + 3] = fmaf(-gm, dv[mm][w4].w, r[4 * w4 + 3]);
                    }
                  }
              }
#pragma unroll
              for (int w4 = 0; w4 < 6; ++w4) {
                r[4 * w4 + 0] = fmaf(-gt, dj[w4].x, r[4 * w4 + 0]);
                r[4 * w4 + 1] = fmaf(-gt, dj[w4].y, r[4 * w4 + 1]);
                r[4 * w4 + 2] = fmaf(-gt, dj[w4].z, r[4 * w4 + 2]);
                r[4 * w4 + 3] = fmaf(-gt, dj[w4].w, r[4 * w4 + 3]);
              }
              t = T + 1;
              float pr = 0.f;
#pragma unroll
              for (int q = 0; q < 24; ++q) pr = fmaf(r[q], r[q], pr);
              rn2 = pair_sum(pr);
              if (it + 1 < s) {
                float inv = 1.f;
                if constexpr (PREC == 2) {
                  float mx = 0.f;
#pragma unroll
                  for (int q = 0; q < 24; ++q) mx = fmaxf(mx, fabsf(r[q]));
                  mx = pair_max(mx);
                  inv = mx > 0.f ? FP8_MAX / mx : 1.f;
                }
                if (wait_staging(job_index(g, k, it + 1)))
                  write_a_part24<PREC>(A, R2, u, r, inv);
                else
                  ok = false;
              }
              if constexpr (PREC != 0) {
#pragma unroll
                for (int q = 0; q < 24; ++q) rsm[q * PGT + gtid] = r[q];
              }
            };
            if (t < 8)
              with_t<8>(t, step);
            else
              active = false;
          }
        }
        fence_proxy_async_smem();
        if (named_bar_or(gbar, PGT, !ok)) {
          ok = false;
          break;
        }
        if (it + 1 < s && gtid == 0) mbar_arrive(&bar_a[g]);
      }
      if (!ok) break;
      if (R2 < rows) {
        const int64_t gi = g0 + R2;
        for (int mm = u; mm < s; mm += 2) {
          a.idx[gi * s + mm] = mm < t ? static_cast<uint16_t>(sel[mm * TILE_M + R2]) : static_cast<uint16_t>(0);
          a.coef[gi * s + mm] = mm < t ? gs[mm * TILE_M + R2] : 0.f;
        }
        if (u == 0) {
          a.nnz[gi] = static_cast<uint8_t>(t);
          if (a.resid_sq) a.resid_sq[gi] = rn2;
        }
      }
    }
#undef LS
#undef IDG
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}
