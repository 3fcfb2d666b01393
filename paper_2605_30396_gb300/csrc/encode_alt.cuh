// Batch-OMP, FP32 (3xTF32) correlations, s <= 8: two tiles per CTA served by
// the same sixteen warps in alternation (Sec. 2.1: OMP against the dictionary,
// one greedy atom at a time, least-squares re-fit).
//
// Included by encode.cu inside namespace dlsh::enc, after encode_pair.cuh
// (it shares that file's staging protocol and MMA helpers).
//
// The warps select for tile A while the tensor pipe computes A's correlations,
// then solve for A while the tensor pipe already computes tile B's; then they
// select for B, solve for B (the tensor pipe on A's next iteration), and so on.
// The one-tile encoder leaves the tensor pipe idle during every solve; here it
// idles only when the accumulator buffers are full.
//   warp 17  TMA producer: 128-atom chunks of the packed dictionary (the
//            one-tile encoder's image), in the MMA warp's order.
//   warp 16  MMA issuer: jobs (tile A, iteration it), (tile B, it), (A, it+1)..;
//            once the previous job's MMAs are done, each job copies its staged
//            residual (TF32 hi, lo) into the tensor-memory A columns, then runs
//            the 3xTF32 MMAs (M = 128, N = 128) of every chunk.
//   warps 0-15  selection (four threads per row, a 32-column quarter of each
//            chunk) and solver (four sub-lanes of 12 interleaved dims per signal), as in
//            the one-tile encoder, on the two tiles in turn.
// Tensor memory: A (hi then lo) in columns 0..95, three 128-column accumulator
// buffers in 128..511, used in job order.  N = 64 MMAs measured at about half
// the throughput of N = 128 ones, so the chunks stay 128 atoms wide.

constexpr int ABN = 128;     // atoms per chunk

constexpr int ABUF = 3;      // accumulator buffers
constexpr int AQC = 32;      // chunk columns read by one selection thread
// K-block stride of the staged A operand: 128 rows of 16 bytes plus 32 bytes of
// skew, so that the 16-byte stores of a quarter-warp (two rows, four K blocks)
// fall on eight different bank groups
constexpr uint32_t ALBO = TILE_M * 16 + 32;
constexpr uint32_t APART = 12 * ALBO;  // the TF32 hi part, then the lo part

struct AltPlan {
  int K, Kp, nchunks, stages, s;
  uint32_t chunk_bytes, a_bytes;
  uint32_t off_stage, off_L[2], off_sel[2], off_y[2], off_cand, off_bar, off_ring, smem;
};

struct AltArgs {
  const float* X;
  int64_t N;
  const float* D32p;
  const float* G;
  const uint8_t* img;
  uint16_t* idx;
  float* coef;
  uint8_t* nnz;
  float* resid_sq;
  float eps;
  uint32_t* status;
  long long budget;
  const long long* n_dev;
  unsigned long long* prof;  // optional: per-phase SM cycles (10 counters)
  AltPlan p;
};

inline int make_alt_plan(int K, int s, int code, AltPlan& p, int smem_limit = SMEM_LIMIT) {
  int top4 = 0;
  if (s > 8 || operand_precision(code, &top4) != 0) return DLSH_ERR_UNSUPPORTED;
  p.K = K;
  p.s = s;
  p.nchunks = (K + ABN - 1) / ABN;
  p.Kp = p.nchunks * ABN;
  p.a_bytes = 2 * APART;
  p.chunk_bytes = ABN * op_kb(0) * 16 * op_parts(0);
  uint32_t off = 0;
  auto take = [&](uint32_t bytes) {
    uint32_t o = (off + 1023u) & ~1023u;
    off = o + bytes;
    return o;
  };
  p.off_stage = take(p.a_bytes);
  // per tile: the factor (its diagonal holds the reciprocals), the support and
  // y; the coefficients go to global memory at every step
  for (int t = 0; t < 2; ++t) {
    p.off_L[t] = take(36 * TILE_M * 4);
    p.off_sel[t] = take(8 * TILE_M * 4);
    p.off_y[t] = take(8 * TILE_M * 4);
  }
  p.off_cand = take(TILE_M * 4 * 8);
  p.off_bar = take(1024);
  const uint32_t fixed = (off + 1023u) & ~1023u;
  if (fixed >= static_cast<uint32_t>(smem_limit)) return DLSH_ERR_UNSUPPORTED;
  int fit = static_cast<int>((smem_limit - fixed) / p.chunk_bytes);
  if (fit > 32) fit = 32;
  if (fit < 2) return DLSH_ERR_UNSUPPORTED;
  p.stages = fit;
  p.off_ring = fixed;
  p.smem = fixed + p.stages * p.chunk_bytes;
  return DLSH_OK;
}

// Sub-lane u of a row owns the dimensions 16k + 4u .. 16k + 4u + 3 (k = 0, 1,
// 2): the four sub-lanes of a row read 16 contiguous bytes of each group, so a
// warp's load touches one cache line per row where the 12-contiguous split
// touched two.
__device__ __forceinline__ int alt_dim(int u, int q) { return 16 * (q >> 2) + 4 * u + (q & 3); }

// Sub-lane u's 12 values (TF32 hi, lo) into the A operand: dims 16k + 4u .. are
// K block 4k + u.
__device__ __forceinline__ void write_a_alt(uint8_t* A, int row, int u, const float (&r)[12]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int kb = 4 * k + u;
    float4 hi, lo;
    hi.x = to_tf32(r[4 * k + 0]);
    hi.y = to_tf32(r[4 * k + 1]);
    hi.z = to_tf32(r[4 * k + 2]);
    hi.w = to_tf32(r[4 * k + 3]);
    lo.x = to_tf32(r[4 * k + 0] - hi.x);
    lo.y = to_tf32(r[4 * k + 1] - hi.y);
    lo.z = to_tf32(r[4 * k + 2] - hi.z);
    lo.w = to_tf32(r[4 * k + 3] - hi.w);
    *reinterpret_cast<float4*>(A + kb * ALBO + row * 16) = hi;
    *reinterpret_cast<float4*>(A + APART + kb * ALBO + row * 16) = lo;
  }
}

// The FP16-split form of the same operand (the split encoder's F16 variant):
// the residual of a row scaled by a power of two, as FP16 hi and lo parts in
// K blocks of 8 elements.  Sub-lane u's dims 16k + 4u .. 16k + 4u + 3 are the
// half (u & 1) of K block 2k + (u >> 1).  A K-block stride of 2048 + 64 bytes
// puts the 8-byte stores of a half-warp (four rows, four sub-lanes) on sixteen
// different bank pairs.
constexpr uint32_t ALBO16 = TILE_M * 16 + 64;
constexpr uint32_t APART16 = 6 * ALBO16;
__device__ __forceinline__ void write_a_f16(uint8_t* A, int row, int u, const float (&r)[12], float scale) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint32_t off = static_cast<uint32_t>(2 * k + (u >> 1)) * ALBO16 + row * 16 + (u & 1) * 8;
    uint2 ph, pl;
    split_f16x4(r[4 * k] * scale, r[4 * k + 1] * scale, r[4 * k + 2] * scale, r[4 * k + 3] * scale, ph, pl);
    *reinterpret_cast<uint2*>(A + off) = ph;
    *reinterpret_cast<uint2*>(A + APART16 + off) = pl;
  }
}

// Passes P0..P1-1 of one chunk of 3xFP16 MMAs (A hi, lo in tensor-memory
// columns 0..23, 24..47; N = 128): pass 0 hi.hi, pass 1 hi.lo(D), pass 2 lo.hi.
template <int P0, int P1>
__device__ __forceinline__ void issue_f16_passes(uint32_t tmem_d, uint32_t a_tmem, uint32_t b_addr) {
  constexpr uint32_t idesc = umma_idesc(0, 0, TILE_M, ABN);
  constexpr uint32_t B_LBO = ABN * 16, SBO = 128, B_PART = ABN * 6 * 16;
#pragma unroll
  for (int pass = P0; pass < P1; ++pass) {
    const uint32_t ao = pass == 2 ? 24u : 0u;
    const uint32_t bo = pass == 1 ? B_PART : 0u;
#pragma unroll
    for (int ks = 0; ks < 3; ++ks) {
      const uint64_t bd = umma_smem_desc(b_addr + bo + ks * 2 * B_LBO, B_LBO, SBO);
      umma_f16_tmem_a(tmem_d, a_tmem + ao + ks * 8, bd, idesc, (pass | ks) != 0);
    }
  }
}

// Passes P0..P1-1 of one chunk of 3xTF32 MMAs, A (hi, lo) from tensor memory,
// N = 128: pass 0 hi(r).hi(D), pass 1 hi(r).lo(D), pass 2 lo(r).hi(D).
template <int P0, int P1>
__device__ __forceinline__ void issue_alt_passes(uint32_t tmem_d, uint32_t a_tmem, uint32_t b_addr) {
  constexpr uint32_t idesc = umma_idesc(2, 2, TILE_M, ABN);
  constexpr uint32_t B_LBO = ABN * 16, SBO = 128, B_PART = ABN * 12 * 16;
#pragma unroll
  for (int pass = P0; pass < P1; ++pass) {
    const uint32_t ao = pass == 2 ? 48u : 0u;
    const uint32_t bo = pass == 1 ? B_PART : 0u;
#pragma unroll
    for (int ks = 0; ks < 6; ++ks) {
      const uint64_t bd = umma_smem_desc(b_addr + bo + ks * 2 * B_LBO, B_LBO, SBO);
      umma_tf32_tmem_a(tmem_d, a_tmem + ao + ks * 8, bd, idesc, (pass | ks) != 0);
    }
  }
}

// Barriers and shared state of the dictionary producer and the MMA issuer,
// shared by the two-tile FP32 encoders.
struct AltSync {
  uint64_t* bar_a;       // [slots] a tile slot's A operand is staged
  uint64_t* bar_full;    // [ABUF] an accumulator buffer holds a chunk's correlations
  uint64_t* bar_empty;   // [ABUF] an accumulator buffer has been read
  uint64_t* bar_stage;   // the staged A operand has been copied into tensor memory
  uint64_t* bar_dfull;   // [stages] a dictionary chunk has landed in the ring
  uint64_t* bar_dempty;  // [stages] the MMAs have finished with a ring stage
  volatile long long* stage_done;  // the last job whose A copy has completed
  unsigned long long* pcs;         // optional phase counters (6..9 are written here), or null
};

// One elected thread: chunk c of the packed dictionary image for every job, in
// job order, through the ring; then waits until the MMAs have released the
// last stages, so that no copy is in flight when the CTA exits.
__device__ __forceinline__ void alt_produce(const AltSync& y, const uint8_t* img, uint8_t* ring, int stages,
                                            uint32_t chunk_bytes, int nchunks, long long njobs,
                                            uint32_t* status, long long budget) {
  long long n = 0;
  int st = 0;
  uint32_t par = 1u;  // bar_dempty parity to wait for at stage st
  bool ok = true;
  for (long long j = 0; j < njobs && ok; ++j)
    for (int c = 0; c < nchunks; ++c, ++n) {
      if (!mbar_wait(&y.bar_dempty[st], par, budget)) {
        flag_status(status, ST_TIMEOUT);
        ok = false;
        break;
      }
      mbar_arrive_expect_tx(&y.bar_dfull[st], chunk_bytes);
      bulk_g2s(ring + static_cast<size_t>(st) * chunk_bytes, img + static_cast<size_t>(c) * chunk_bytes,
               chunk_bytes, &y.bar_dfull[st]);
      if (++st == stages) {
        st = 0;
        par ^= 1u;
      }
    }
  for (long long f = n > stages ? n - stages : 0; ok && f < n; ++f) {
    if (!mbar_wait(&y.bar_dempty[f % stages], static_cast<uint32_t>((f / stages) & 1), budget)) {
      flag_status(status, ST_TIMEOUT);
      ok = false;
    }
  }
}

// One elected thread: the jobs (slot 0, it), (slot 1, it), .., (slot 0, it + 1)
// .. of the rounds k (slot t has a tile in rounds k < Kt[t], Kt non-increasing)
// of s iterations.  Each job waits for its staged residual,
// for the previous job's MMAs (the A columns in tensor memory are shared),
// copies the hi / lo residual into tensor memory (TF32: columns 0..95; F16:
// 0..47), then runs the three-product MMAs of every chunk into the
// accumulator buffers in turn.
template <bool F16, int NS>
__device__ __forceinline__ void alt_issue(const AltSync& y, uint32_t tmem_base, uint32_t acc0, uint32_t stage_addr,
                                          uint32_t ring_addr, int stages, uint32_t chunk_bytes, int nchunks,
                                          const int (&Kt)[NS], int s, uint32_t* status, long long budget) {
  unsigned long long* pcs = y.pcs;
  uint32_t aph[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) aph[t] = 0u;
  long long job = 0;
  // the next chunk's ring stage and accumulator buffer with the parities of
  // their bar_dfull / bar_full phases; the previous chunk's buffer
  int st = 0, buf = 0, lbuf = -1;
  uint32_t dpar = 0u, fpar = 0u, lfpar = 0u;
  bool ok = true;
  auto fail = [&]() {
    flag_status(status, ST_TIMEOUT);
    ok = false;
  };
  // the next chunk's resources: its dictionary chunk has landed and its
  // accumulator buffer has been read
  auto wait_chunk = [&]() -> bool {
    const long long W2 = pcs ? clock64() : 0;
    const bool okd = mbar_wait(&y.bar_dfull[st], dpar, budget);
    const long long W3 = pcs ? clock64() : 0;
    const bool oke = okd && mbar_wait(&y.bar_empty[buf], fpar ^ 1u, budget);
    if (pcs) {
      pcs[7] += W3 - W2;
      pcs[8] += clock64() - W3;
    }
    return oke;
  };
  for (int k = 0; k < Kt[0] && ok; ++k) {
    int nk = 0;  // slots with a tile in round k
#pragma unroll
    for (int t = 0; t < NS; ++t) nk += k < Kt[t];
    for (int it = 0; it < s && ok; ++it)
      for (int t = 0; t < nk && ok; ++t, ++job) {
        const long long W0 = pcs ? clock64() : 0;
        if (!mbar_wait(&y.bar_a[t], aph[t], budget)) {
          fail();
          break;
        }
        if (pcs) pcs[6] += clock64() - W0;
        aph[t] ^= 1u;
        if (lbuf >= 0 && !mbar_wait(&y.bar_full[lbuf], lfpar, budget)) {
          fail();
          break;
        }
        tc_fence_after();
        {
          constexpr uint32_t SBO = 128;
          if constexpr (F16) {
#pragma unroll
            for (int part = 0; part < 2; ++part)
#pragma unroll
              for (int kk = 0; kk < 3; ++kk)
                tmem_cp_128x256b(tmem_base + part * 24 + kk * 8,
                                 umma_smem_desc(stage_addr + part * APART16 + kk * 2 * ALBO16, ALBO16, SBO));
          } else {
#pragma unroll
            for (int part = 0; part < 2; ++part)
#pragma unroll
              for (int kk = 0; kk < 6; ++kk)
                tmem_cp_128x256b(tmem_base + part * 48 + kk * 8,
                                 umma_smem_desc(stage_addr + part * APART + kk * 2 * ALBO, ALBO, SBO));
          }
          tc_commit(y.bar_stage);
          const long long W1 = pcs ? clock64() : 0;
          if (!mbar_wait(y.bar_stage, static_cast<uint32_t>(job & 1), budget)) {
            fail();
            break;
          }
          if (pcs) pcs[9] += clock64() - W1;
          *y.stage_done = job;
        }
        if (!wait_chunk()) {
          fail();
          break;
        }
        for (int c = 0; c < nchunks; ++c) {
          tc_fence_after();
          const uint32_t d = tmem_base + acc0 + static_cast<uint32_t>(buf) * ABN;
          const uint32_t b = ring_addr + static_cast<uint32_t>(st) * chunk_bytes;
          if constexpr (F16)
            issue_f16_passes<0, 2>(d, tmem_base, b);
          else
            issue_alt_passes<0, 2>(d, tmem_base, b);
          // the next chunk's resources are checked while the last pass of
          // this one runs, so the checks do not leave the tensor pipe idle
          const int cst = st, cbuf = buf;
          lbuf = buf;
          lfpar = fpar;
          if (++st == stages) {
            st = 0;
            dpar ^= 1u;
          }
          if (++buf == ABUF) {
            buf = 0;
            fpar ^= 1u;
          }
          const bool nok = c + 1 < nchunks ? wait_chunk() : true;
          if constexpr (F16)
            issue_f16_passes<2, 3>(d, tmem_base, b);
          else
            issue_alt_passes<2, 3>(d, tmem_base, b);
          tc_commit(&y.bar_full[cbuf]);
          tc_commit(&y.bar_dempty[cst]);
          if (!nok) {
            fail();
            break;
          }
        }
      }
  }
}

// (a template only so that the header can be included by several translation
// units; instantiated in enc_split.cu)
template <int V = 0>
__global__ void __launch_bounds__(NTHREADS, 1) encode_alt_kernel(const __grid_constant__ AltArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr uint32_t ACC0 = 128;
  const AltPlan& p = a.p;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long NS = a.n_dev ? *a.n_dev : a.N;
  const int ntiles = static_cast<int>((NS + TILE_M - 1) / TILE_M);
  const int Gd = static_cast<int>(gridDim.x), bidx = static_cast<int>(blockIdx.x);
  const int s = p.s;
  // rounds k in which tile slot 0 / slot 1 have a tile (tiles b + (2k + slot) Gd)
  const int K0 = bidx < ntiles ? (ntiles - bidx + 2 * Gd - 1) / (2 * Gd) : 0;
  const int K1 = bidx + Gd < ntiles ? (ntiles - bidx - Gd + 2 * Gd - 1) / (2 * Gd) : 0;
  auto job_index = [&](int t, int k, int it) -> long long {
    return k < K1 ? 2LL * s * k + 2LL * it + t : 2LL * s * K1 + static_cast<long long>(s) * (k - K1) + it;
  };

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + p.off_bar);
  uint64_t* bar_a = bars;            // [2]
  uint64_t* bar_full = bars + 2;     // [ABUF]
  uint64_t* bar_empty = bars + 5;    // [ABUF]
  uint64_t* bar_stage = bars + 8;
  uint64_t* bar_dfull = bars + 9;    // [stages]
  uint64_t* bar_dempty = bar_dfull + p.stages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_dempty + p.stages);
  volatile long long* stage_done = reinterpret_cast<volatile long long*>(smem + p.off_bar + 1000);
  // optional phase profile, SM cycles: 0 selection waiting for MMAs, 1 selection
  // (incl. 0), 2 solver, 3 solver waiting for the staging area, 4 tile
  // iterations (thread 0); 6 MMA warp waiting for a residual, 7 for a
  // dictionary chunk, 8 for an accumulator buffer, 9 for the copy into TMEM
  unsigned long long* pcs = reinterpret_cast<unsigned long long*>(smem + p.off_bar + 512);
  const bool prof_any = a.prof != nullptr;

  if (tid == 0) {
    mbar_init(&bar_a[0], 1);
    mbar_init(&bar_a[1], 1);
    for (int b = 0; b < ABUF; ++b) {
      mbar_init(&bar_full[b], 1);
      mbar_init(&bar_empty[b], NEPI / 32);
    }
    mbar_init(bar_stage, 1);
    for (int q = 0; q < p.stages; ++q) {
      mbar_init(&bar_dfull[q], 1);
      mbar_init(&bar_dempty[q], 1);
    }
    *stage_done = -1;
    if (prof_any)
      for (int q = 0; q < 10; ++q) pcs[q] = 0;
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

  const AltSync sy{bar_a, bar_full, bar_empty, bar_stage, bar_dfull, bar_dempty, stage_done, prof_any ? pcs : nullptr};
  if (warp == NEPI / 32 + 1) {
    // ------------------------------------------------ TMA producer
    if (lane == 0)
      alt_produce(sy, a.img, smem + p.off_ring, p.stages, p.chunk_bytes, p.nchunks,
                  static_cast<long long>(s) * (K0 + K1), a.status, a.budget);
  } else if (warp == NEPI / 32) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0)
      alt_issue<false, 2>(sy, tmem_base, ACC0, smem_u32(smem + p.off_stage), ring_addr, p.stages, p.chunk_bytes,
                          p.nchunks, {K0, K1}, s, a.status, a.budget);
  } else {
    // ------------------------------------------------ selection + solver, two tiles in turn
    uint8_t* A = smem + p.off_stage;
    float* cv = reinterpret_cast<float*>(smem + p.off_cand);  // [128][4]
    int* cj = reinterpret_cast<int*>(smem + p.off_cand + TILE_M * 4 * 4);
    const int R1 = 32 * (warp & 3) + lane, q1 = warp >> 2;
    const int R2 = 8 * warp + (lane >> 2), u = lane & 3;
    const uint32_t trow = tmem_base + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + ACC0 +
                          static_cast<uint32_t>(q1 * AQC);
    const int K = p.K, nchunks = p.nchunks;
    const float eps2 = a.eps * a.eps;
    int sbuf = 0;       // accumulator buffer of the next chunk
    uint32_t spar = 0u;  // and the parity of its bar_full phase
    bool ok = true;
    // the staging area may be written for job J once the copy of job J - 1 has
    // completed (published by the MMA warp)
    auto wait_staging = [&](long long J) -> bool {
      const long long t0 = clock64();
      while (*stage_done < J - 1) {
        if (clock64() - t0 > a.budget) {
          flag_status(a.status, ST_TIMEOUT);
          return false;
        }
      }
      return true;
    };
    // sub-lane u's 12 dims of row R2 of tile `tl` into the staging area; the
    // row's ||x||^2
    auto stage_x = [&](long long tl) -> float {
      const int64_t tg0 = tl * TILE_M;
      const bool tin = R2 < (NS - tg0 < TILE_M ? NS - tg0 : TILE_M);
      const float* txr = a.X + (tg0 + R2) * DLSH_D;
      float x[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) x[q] = (tin && alt_dim(u, q) < DLSH_D) ? __ldg(txr + alt_dim(u, q)) : 0.f;
      float part = 0.f;
#pragma unroll
      for (int q = 0; q < 12; ++q) part = fmaf(x[q], x[q], part);
      write_a_alt(A, R2, u, x);
      return quad_sum(part);
    };
    auto tile_of = [&](int t, int k) -> long long { return static_cast<long long>(bidx) + (2LL * k + t) * Gd; };
    // per-tile state of this thread's row (R2) in each slot
    // (two named copies, so that the loop over the tiles need not be unrolled)
    float rn2_0 = 0.f, rn2_1 = 0.f, xn_0 = 0.f, xn_1 = 0.f;
    bool act_0 = false, act_1 = false;
    int tc_0 = 0, tc_1 = 0;
    // -------- the first round's signals: slot 0, then (once its copy is done) slot 1
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if ((t == 0 ? K0 : K1) > 0 && ok) {
        if (!wait_staging(job_index(t, 0, 0))) ok = false;
        if (ok) {
          const float v = stage_x(tile_of(t, 0));
          if (t == 0) rn2_0 = v; else rn2_1 = v;
        }
        fence_proxy_async_smem();
        if (named_bar_or(1, NEPI, !ok)) ok = false;
        if (ok && tid == 0) mbar_arrive(&bar_a[t]);
      }
    }
    for (int k = 0; k < K0 && ok; ++k) {
      const bool two = k < K1;
      {
        const long long tl0 = tile_of(0, k), tl1 = tile_of(1, k);
        const int rows0 = static_cast<int>(NS - tl0 * TILE_M < TILE_M ? NS - tl0 * TILE_M : TILE_M);
        const int rows1 = static_cast<int>(NS - tl1 * TILE_M < TILE_M ? NS - tl1 * TILE_M : TILE_M);
        xn_0 = sqrtf(rn2_0);
        xn_1 = sqrtf(rn2_1);
        act_0 = R2 < rows0;
        act_1 = two && R2 < rows1;
        tc_0 = tc_1 = 0;
      }
      for (int it = 0; it < s && ok; ++it) {
#pragma unroll 1
        for (int t = 0; t < (two ? 2 : 1); ++t) {
          float rn2c = t ? rn2_1 : rn2_0;
          const float xnc = t ? xn_1 : xn_0;
          bool actc = t ? act_1 : act_0;
          int tcc = t ? tc_1 : tc_0;
          float* Ls = reinterpret_cast<float*>(smem + p.off_L[t]);
          int* sel = reinterpret_cast<int*>(smem + p.off_sel[t]);
          float* ys = reinterpret_cast<float*>(smem + p.off_y[t]);
#define LS(rr, cc2) Ls[(((rr) * ((rr) + 1)) / 2 + (cc2)) * TILE_M + R2]
#define IDG(rr) LS(rr, rr)
          const long long tl = tile_of(t, k);
          const int64_t g0 = tl * TILE_M;
          const int rows = static_cast<int>(NS - g0 < TILE_M ? NS - g0 : TILE_M);
          const bool in_tile = R2 < rows;
          const float* xr = a.X + (g0 + R2) * DLSH_D;
          // ================= phase 1: selection over this thread's column quarter
          const bool prof_on = prof_any && tid == 0;
          const long long T0 = prof_on ? clock64() : 0;
          {
            uint32_t best = 0;
            int bestc = 0;
            for (int c = 0; c < nchunks; ++c) {
              const int buf = sbuf;
              const uint32_t spar0 = spar;
              if (++sbuf == ABUF) {
                sbuf = 0;
                spar ^= 1u;
              }
              const long long W4 = prof_on ? clock64() : 0;
              if (!mbar_wait(&bar_full[buf], spar0, a.budget)) {
                flag_status(a.status, ST_TIMEOUT);
                ok = false;
                break;
              }
              if (prof_on) pcs[0] += clock64() - W4;
              tc_fence_after();
              __syncwarp();
              uint32_t rr[AQC];
              tmem_ld32_issue(trow + static_cast<uint32_t>(buf * ABN), rr);
              tmem_ld32_wait(rr);
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&bar_empty[buf]);
              uint32_t m0 = 0, m1 = 0;
#pragma unroll
              for (int q = 0; q < AQC; q += 2) {
                m0 = max(m0, (rr[q] & 0x7fffffe0u) | static_cast<uint32_t>(31 - q));
                m1 = max(m1, (rr[q + 1] & 0x7fffffe0u) | static_cast<uint32_t>(30 - q));
              }
              const uint32_t m = max(m0, m1);
              if ((m & ~31u) > (best & ~31u)) {
                best = m;
                bestc = c;
              }
            }
            cv[R1 * 4 + q1] = __uint_as_float(best & ~31u);
            cj[R1 * 4 + q1] = bestc * ABN + q1 * AQC + 31 - static_cast<int>(best & 31u);
          }
          if (named_bar_or(1, NEPI, !ok)) {
            ok = false;
            break;
          }
          const long long T1 = prof_on ? clock64() : 0;
          // ================= phase 2: merge, Cholesky, solve, residual
          const int tt = tcc;
          bool act = actc;
          if (act && rn2c <= eps2) act = false;
          if (act) {
            // the step for a support of tt atoms, compiled once per tt
            auto step = [&](auto tag) {
              constexpr int T = decltype(tag)::value;
              constexpr int TA = T > 0 ? T : 1;
              float x[12], r[12];
#pragma unroll
              for (int q = 0; q < 12; ++q) x[q] = (in_tile && alt_dim(u, q) < DLSH_D) ? __ldg(xr + alt_dim(u, q)) : 0.f;
              int sl[TA];
#pragma unroll
              for (int m = 0; m < T; ++m) sl[m] = sel[m * TILE_M + R2];
              int js = -1;
              float bestv = -1.f;
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                const float v = cv[R2 * 4 + qq];
                const int j = cj[R2 * 4 + qq];
                if (j < K && (v > bestv || (v == bestv && j < js))) {
                  bestv = v;
                  js = j;
                }
              }
              bool dup = false;
#pragma unroll
              for (int m = 0; m < T; ++m) dup |= sl[m] == js;
              if (dup) js = -1;
              if (js < 0 || !(bestv > CORR_STOP_REL * xnc)) {
                act = false;
                return;
              }
              const float* Grow = a.G + static_cast<size_t>(js) * K;
              float gv[TA];
#pragma unroll
              for (int m = 0; m < T; ++m) gv[m] = __ldg(Grow + sl[m]);
              const float gjj = __ldg(Grow + js);
              float4 dj[3];
              {
                const float4* dr = reinterpret_cast<const float4*>(a.D32p + static_cast<size_t>(js) * DPAD + 4 * u);
#pragma unroll
                for (int w4 = 0; w4 < 3; ++w4) dj[w4] = __ldg(dr + 4 * w4);
              }
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
                act = false;
                return;
              }
              const float ell = sqrtf(ell2);
              const float iell = 1.f / ell;
#pragma unroll
              for (int m = 0; m < T; ++m) LS(T, m) = w[m];
              IDG(T) = iell;  // the diagonal holds 1 / L(t, t)
              float bp = 0.f;
#pragma unroll
              for (int w4 = 0; w4 < 3; ++w4) {
                bp = fmaf(dj[w4].x, x[4 * w4 + 0], bp);
                bp = fmaf(dj[w4].y, x[4 * w4 + 1], bp);
                bp = fmaf(dj[w4].z, x[4 * w4 + 2], bp);
                bp = fmaf(dj[w4].w, x[4 * w4 + 3], bp);
              }
              float yv[TA];
#pragma unroll
              for (int m = 0; m < T; ++m) yv[m] = ys[m * TILE_M + R2];
              float yt = quad_sum(bp);
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
              // the row's coefficients so far (sub-lane u writes slots u, u+4)
              {
                const int64_t gi = g0 + R2;
#pragma unroll
                for (int m = 0; m < T; ++m)
                  if ((m & 3) == u) a.coef[gi * s + m] = gam[m];
                if ((T & 3) == u) a.coef[gi * s + T] = gt;
              }
#pragma unroll
              for (int q = 0; q < 12; ++q) r[q] = x[q];
              // the support atoms' rows in groups of up to four, all loads of a
              // group issued before its FMAs (one L2 round trip per group)
#pragma unroll
              for (int m0 = 0; m0 < T; m0 += 4) {
                float4 dv[4][3];
#pragma unroll
                for (int mm = 0; mm < 4; ++mm)
                  if (m0 + mm < T) {
                    const float4* da =
                        reinterpret_cast<const float4*>(a.D32p + static_cast<size_t>(sl[m0 + mm]) * DPAD + 4 * u);
#pragma unroll
                    for (int w4 = 0; w4 < 3; ++w4) dv[mm][w4] = __ldg(da + 4 * w4);
                  }
#pragma unroll
                for (int mm = 0; mm < 4; ++mm)
                  if (m0 + mm < T) {
                    const float gm = gam[m0 + mm];
#pragma unroll
                    for (int w4 = 0; w4 < 3; ++w4) {
                      r[4 * w4 + 0] = fmaf(-gm, dv[mm][w4].x, r[4 * w4 + 0]);
                      r[4 * w4 + 1] = fmaf(-gm, dv[mm][w4].y, r[4 * w4 + 1]);
                      r[4 * w4 + 2] = fmaf(-gm, dv[mm][w4].z, r[4 * w4 + 2]);
                      r[4 * w4 + 3] = fmaf(-gm, dv[mm][w4].w, r[4 * w4 + 3]);
                    }
                  }
              }
#pragma unroll
              for (int w4 = 0; w4 < 3; ++w4) {
                r[4 * w4 + 0] = fmaf(-gt, dj[w4].x, r[4 * w4 + 0]);
                r[4 * w4 + 1] = fmaf(-gt, dj[w4].y, r[4 * w4 + 1]);
                r[4 * w4 + 2] = fmaf(-gt, dj[w4].z, r[4 * w4 + 2]);
                r[4 * w4 + 3] = fmaf(-gt, dj[w4].w, r[4 * w4 + 3]);
              }
              tcc = T + 1;
              float pr = 0.f;
#pragma unroll
              for (int q = 0; q < 12; ++q) pr = fmaf(r[q], r[q], pr);
              rn2c = quad_sum(pr);
              if (it + 1 < s) {
                const long long W5 = prof_on ? clock64() : 0;
                if (wait_staging(job_index(t, k, it + 1)))
                  write_a_alt(A, R2, u, r);
                else
                  ok = false;
                if (prof_on) pcs[3] += clock64() - W5;
              }
            };
            if (tt < 8)
              with_t<8>(tt, step);
            else
              act = false;
          }
          actc = act;
          // last iteration: write this slot's codes, then stage its next tile's
          // signals (the MMA warp needs them right after the other slot's job)
          if (it + 1 == s) {
            if (in_tile) {
              const int64_t gi = g0 + R2;
              const int tn = tcc;
              for (int mm = u; mm < s; mm += 4) {
                a.idx[gi * s + mm] = mm < tn ? static_cast<uint16_t>(sel[mm * TILE_M + R2]) : static_cast<uint16_t>(0);
                if (mm >= tn) a.coef[gi * s + mm] = 0.f;
              }
              if (u == 0) {
                a.nnz[gi] = static_cast<uint8_t>(tn);
                if (a.resid_sq) a.resid_sq[gi] = rn2c;
              }
            }
            if (k + 1 < (t == 0 ? K0 : K1) && ok) {
              if (wait_staging(job_index(t, k + 1, 0)))
                rn2c = stage_x(tile_of(t, k + 1));
              else
                ok = false;
            }
          }
          fence_proxy_async_smem();
          if (named_bar_or(1, NEPI, !ok)) {
            ok = false;
            break;
          }
          const bool more = it + 1 < s || k + 1 < (t == 0 ? K0 : K1);
          if (more && tid == 0) mbar_arrive(&bar_a[t]);
          if (prof_on) {
            pcs[1] += T1 - T0;
            pcs[2] += clock64() - T1;
            pcs[4] += 1;
          }
          if (t == 0) {
            rn2_0 = rn2c;
            act_0 = actc;
            tc_0 = tcc;
          } else {
            rn2_1 = rn2c;
            act_1 = actc;
            tc_1 = tcc;
          }
#undef LS
#undef IDG
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (prof_any && tid == 0) {
    for (int q = 0; q < 10; ++q) atomicAdd(a.prof + q, pcs[q]);
    if (blockIdx.x == 0) a.prof[11] = 3;  // the variant that ran: two tiles served in turn
  }
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}
