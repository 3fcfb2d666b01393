// Batch-OMP, FP32 correlations (three TF32 or three FP16 products), s <= 8:
// two or three tiles per CTA with the warps split by task (Sec. 2.1: OMP against the dictionary, one greedy atom at
// a time, least-squares re-fit).
//
// Included by encode.cu inside namespace dlsh::enc, after encode_alt.cuh (it
// uses that file's dictionary producer, MMA issuer, A-operand layout and the
// staging protocol).
//
// In the alternating encoder all sixteen warps select and then solve, so the
// ALU-bound argmax and the load-bound solver never run at the same time, and
// the selection waits for the MMAs of its own tile.  Here
//   warps 0-7   select: warp w reads tensor-memory lane quarter w & 3 and the
//               column half w >> 2 of every 128-atom chunk, keeps the largest
//               |c| of each 32-column group, and hands one candidate per row
//               and half to the solver warps;
//   warps 8-15  solve: two passes of 64 rows (four sub-lanes of 12 interleaved
//               dims per row), the Cholesky update, the coefficients and the
//               residual, which they stage as the tile's next A operand;
//   warp 16     issues the MMAs, warp 17 streams the dictionary (as in the
//               alternating encoder).
// The selection warps run ahead of the solver warps: while the solver works on
// tile A's iteration it, the tensor pipe computes and the selection warps
// reduce tile B's correlations.  With two tiles a tile's solver, MMAs and
// selection still form one chain per iteration, so each warp group waits for
// the other part of the time; a third tile (which fits beside the FP16
// operands) lets the solver run two jobs behind the selection.  Per job the
// time is then the largest of the MMAs, the selection and the solver instead
// of the sum of selection and solver.

constexpr int SPW = 8;         // selection warps (0..7)
constexpr int SVT = 256;       // solver threads (warps 8..15)
constexpr int SMAXSLOT = 3;    // tile slots per CTA (2, or 3 with FP16 parts)

struct SplitPlan {
  int K, Kp, nchunks, stages, s;
  uint32_t chunk_bytes, a_bytes;
  // per tile slot: the factor (its diagonal holds the reciprocals), the
  // support, y, the row state (||r||^2, ||x||, atoms taken and a stop bit, the
  // inverse of the staged operand's scale) and the candidates of the selection
  // warps (two per row)
  int nslots;
  uint32_t off_stage, off_L[SMAXSLOT], off_sel[SMAXSLOT], off_y[SMAXSLOT], off_row[SMAXSLOT], off_cand[SMAXSLOT];
  // FP16 parts with two slots: each solver thread's 12 signal values of its
  // rows, kept for the tile's iterations ([12][512] floats per slot)
  uint32_t off_x[SMAXSLOT];
  uint32_t off_bar, off_ring, smem;
};

struct SplitArgs {
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
  unsigned long long* prof;  // optional: per-phase SM cycles (see dlsh.h)
  SplitPlan p;
};

// f16: the correlations as three FP16 products (the operand split into FP16 hi
// and lo parts of a power-of-two scaled copy) instead of three TF32 products;
// nslots: tiles per CTA in flight (2 or 3).
inline int make_split_plan(int K, int s, int code, SplitPlan& p, bool f16, int nslots = 2,
                           int smem_limit = SMEM_LIMIT) {
  int top4 = 0;
  if (s > 8 || operand_precision(code, &top4) != 0 || nslots < 2 || nslots > SMAXSLOT)
    return DLSH_ERR_UNSUPPORTED;
  p.K = K;
  p.s = s;
  p.nslots = nslots;
  p.nchunks = (K + ABN - 1) / ABN;
  p.Kp = p.nchunks * ABN;
  p.a_bytes = f16 ? 2 * APART16 : 2 * APART;
  p.chunk_bytes = f16 ? ABN * 6 * 16 * 2 : ABN * op_kb(0) * 16 * op_parts(0);
  uint32_t off = 0;
  auto take = [&](uint32_t bytes) {
    uint32_t o = (off + 127u) & ~127u;
    off = o + bytes;
    return o;
  };
  p.off_stage = take(p.a_bytes);
  for (int t = 0; t < nslots; ++t) {
    p.off_L[t] = take(36 * TILE_M * 4);
    p.off_sel[t] = take(8 * TILE_M * 4);
    p.off_y[t] = take(8 * TILE_M * 4);
    p.off_row[t] = take(4 * TILE_M * 4);
    p.off_cand[t] = take(2 * TILE_M * 8);
    p.off_x[t] = (f16 && nslots == 2) ? take(12 * 4 * TILE_M * 4) : 0u;
  }
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

template <bool F16, int NSL>
__global__ void __launch_bounds__(NTHREADS, 1) encode_split_kernel(const __grid_constant__ SplitArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr uint32_t ACC0 = 128;
  const SplitPlan& p = a.p;
  // the signals stay in shared memory across a tile's iterations (only the
  // two-slot FP16 layout has room for them)
  constexpr bool XC = F16 && NSL == 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long NS = a.n_dev ? *a.n_dev : a.N;
  const int ntiles = static_cast<int>((NS + TILE_M - 1) / TILE_M);
  const int Gd = static_cast<int>(gridDim.x), bidx = static_cast<int>(blockIdx.x);
  const int s = p.s;
  // rounds k in which tile slot t has a tile (tiles b + (NSL k + t) Gd); the
  // counts do not increase with t
  int Kt[NSL];
#pragma unroll
  for (int t = 0; t < NSL; ++t)
    Kt[t] = bidx + t * Gd < ntiles ? (ntiles - bidx - t * Gd + NSL * Gd - 1) / (NSL * Gd) : 0;
  auto slots_in = [&](int k) -> int {
    int n = 0;
#pragma unroll
    for (int t = 0; t < NSL; ++t) n += k < Kt[t];
    return n;
  };
  // jobs run round by round, iteration by iteration, slot by slot
  auto job_index = [&](int t, int k, int it) -> long long {
    long long before = 0;
#pragma unroll
    for (int q = 0; q < NSL; ++q) before += k < Kt[q] ? k : Kt[q];
    return before * s + static_cast<long long>(it) * slots_in(k) + t;
  };
  auto tile_of = [&](int t, int k) -> long long { return static_cast<long long>(bidx) + (static_cast<long long>(NSL) * k + t) * Gd; };
  auto rounds_of = [&](int t) -> int {
    int r = Kt[0];
#pragma unroll
    for (int q = 1; q < NSL; ++q)
      if (q == t) r = Kt[q];
    return r;
  };
  auto rows_of = [&](long long tl) -> int {
    const long long g0 = tl * TILE_M;
    return static_cast<int>(NS - g0 < TILE_M ? NS - g0 : TILE_M);
  };

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + p.off_bar);
  uint64_t* bar_a = bars;                  // [NSL]
  uint64_t* bar_full = bars + NSL;          // [ABUF]
  uint64_t* bar_empty = bar_full + ABUF;   // [ABUF]
  uint64_t* bar_stage = bar_empty + ABUF;
  uint64_t* cand_full = bar_stage + 1;     // [NSL] the selection warps' candidates of a slot are written
  uint64_t* cand_empty = cand_full + NSL;   // [NSL] the solver warps have read them
  uint64_t* bar_dfull = cand_empty + NSL;   // [stages]
  uint64_t* bar_dempty = bar_dfull + p.stages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_dempty + p.stages);
  volatile long long* stage_done = reinterpret_cast<volatile long long*>(smem + p.off_bar + 1000);
  // optional phase profile, SM cycles: 0 selection waiting for MMAs, 1
  // selection (incl. 0 and 10), 2 solver (incl. 3 and 5), 3 solver waiting for
  // the staging area, 4 jobs, 5 solver waiting for candidates; 6 MMA warp
  // waiting for a residual, 7 for a dictionary chunk, 8 for an accumulator
  // buffer, 9 for the copy into TMEM; 10 selection waiting for the solver to
  // take the previous candidates
  unsigned long long* pcs = reinterpret_cast<unsigned long long*>(smem + p.off_bar + 512);
  const bool prof_any = a.prof != nullptr;

  if (tid == 0) {
    for (int t = 0; t < NSL; ++t) mbar_init(&bar_a[t], 1);
    for (int b = 0; b < ABUF; ++b) {
      mbar_init(&bar_full[b], 1);
      mbar_init(&bar_empty[b], SPW);
    }
    mbar_init(bar_stage, 1);
    for (int t = 0; t < NSL; ++t) {
      mbar_init(&cand_full[t], SPW);
      mbar_init(&cand_empty[t], SVT / 32);
    }
    for (int q = 0; q < p.stages; ++q) {
      mbar_init(&bar_dfull[q], 1);
      mbar_init(&bar_dempty[q], 1);
    }
    *stage_done = -1;
    if (prof_any)
      for (int q = 0; q < 12; ++q) pcs[q] = 0;
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
    if (lane == 0) {
      long long rounds = 0;
#pragma unroll
      for (int t = 0; t < NSL; ++t) rounds += Kt[t];
      alt_produce(sy, a.img, smem + p.off_ring, p.stages, p.chunk_bytes, p.nchunks,
                  static_cast<long long>(s) * rounds, a.status, a.budget);
    }
  } else if (warp == NEPI / 32) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0)
      alt_issue<F16, NSL>(sy, tmem_base, ACC0, smem_u32(smem + p.off_stage), ring_addr, p.stages, p.chunk_bytes,
                         p.nchunks, Kt, s, a.status, a.budget);
  } else if (warp < SPW) {
    // ------------------------------------------------ selection, one job ahead of the solver
    const int wq = warp & 3, h = warp >> 2;
    const int R1 = 32 * wq + lane;
    const uint32_t trow = tmem_base + (static_cast<uint32_t>(32 * wq) << 16) + ACC0 + static_cast<uint32_t>(h * 64);
    const bool prof_on = prof_any && tid == 0;
    int sbuf = 0;         // accumulator buffer of the next chunk
    uint32_t spar = 0u;   // and the parity of its bar_full phase
    uint32_t epar = (1u << NSL) - 1u;  // bit t: cand_empty parity to wait for at slot t (the first pass is free)
    bool ok = true;
    for (int k = 0; k < Kt[0] && ok; ++k)
      for (int it = 0; it < s && ok; ++it)
        for (int t = 0; t < slots_in(k) && ok; ++t) {
          const long long T0 = prof_on ? clock64() : 0;
          // the largest truncated |c| of each 32-column group with its column
          // in the low five bits (31 - column, so that ties keep the smaller
          // column), and the chunk it came from
          uint32_t b0 = 0u, b1 = 0u;
          int c0 = 0, c1 = 0;
          for (int c = 0; c < p.nchunks; ++c) {
            const int buf = sbuf;
            const uint32_t par = spar;
            if (++sbuf == ABUF) {
              sbuf = 0;
              spar ^= 1u;
            }
            const long long W0 = prof_on ? clock64() : 0;
            if (!mbar_wait(&bar_full[buf], par, a.budget)) {
              flag_status(a.status, ST_TIMEOUT);
              ok = false;
              break;
            }
            if (prof_on) pcs[0] += clock64() - W0;
            tc_fence_after();
            __syncwarp();
            uint32_t r0[32], r1[32];
            tmem_ld32_issue(trow + static_cast<uint32_t>(buf * ABN), r0);
            tmem_ld32_issue(trow + static_cast<uint32_t>(buf * ABN + 32), r1);
            tmem_ld32_wait(r0);
            tmem_ld32_wait(r1);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_empty[buf]);
            uint32_t m0 = 0u, m1 = 0u, n0 = 0u, n1 = 0u;
#pragma unroll
            for (int q = 0; q < 32; q += 2) {
              m0 = max(m0, (r0[q] & 0x7fffffe0u) | static_cast<uint32_t>(31 - q));
              m1 = max(m1, (r0[q + 1] & 0x7fffffe0u) | static_cast<uint32_t>(30 - q));
              n0 = max(n0, (r1[q] & 0x7fffffe0u) | static_cast<uint32_t>(31 - q));
              n1 = max(n1, (r1[q + 1] & 0x7fffffe0u) | static_cast<uint32_t>(30 - q));
            }
            const uint32_t m = max(m0, m1), n = max(n0, n1);
            if ((m & ~31u) > (b0 & ~31u)) {
              b0 = m;
              c0 = c;
            }
            if ((n & ~31u) > (b1 & ~31u)) {
              b1 = n;
              c1 = c;
            }
          }
          if (!ok) break;
          // this thread's candidate: the better group, ties to the smaller column
          const float v0 = __uint_as_float(b0 & ~31u), v1 = __uint_as_float(b1 & ~31u);
          const int j0 = c0 * ABN + h * 64 + 31 - static_cast<int>(b0 & 31u);
          const int j1 = c1 * ABN + h * 64 + 32 + 31 - static_cast<int>(b1 & 31u);
          const bool second = v1 > v0 || (v1 == v0 && j1 < j0);
          const long long W1 = prof_on ? clock64() : 0;
          if (!mbar_wait(&cand_empty[t], (epar >> t) & 1u, a.budget)) {
            flag_status(a.status, ST_TIMEOUT);
            ok = false;
            break;
          }
          epar ^= 1u << t;
          if (prof_on) pcs[10] += clock64() - W1;
          float* cv = reinterpret_cast<float*>(smem + p.off_cand[t]);
          int* cj = reinterpret_cast<int*>(smem + p.off_cand[t] + TILE_M * 2 * 4);
          cv[R1 * 2 + h] = second ? v1 : v0;
          cj[R1 * 2 + h] = second ? j1 : j0;
          __syncwarp();
          if (lane == 0) mbar_arrive(&cand_full[t]);
          if (prof_on) pcs[1] += clock64() - T0;
        }
  } else {
    // ------------------------------------------------ solver: two passes of 64 rows per job
    const int vt = tid - SPW * 32, vw = vt >> 5;
    const int u = lane & 3;
    const bool prof_on = prof_any && vt == 0;
    uint8_t* A = smem + p.off_stage;
    const int K = p.K;
    const float eps2 = a.eps * a.eps;
    uint32_t fpar = 0u;  // bit t: cand_full parity to wait for at slot t
    bool ok = true;
    auto row_of = [&](int ps) -> int { return 64 * ps + 8 * vw + (lane >> 2); };
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
    // sub-lane u's 12 values of a row's operand into the staging area.  F16:
    // scaled by 2^e so that the row's largest |value| lies in [2^14, 2^15)
    // (the FP16 parts then keep FP32's 22 significant bits); returns the
    // inverse of the correlations' scale (2^-(e + 8), the dictionary image
    // being 256 D), 1 for TF32
    auto stage_row = [&](int r, const float (&v)[12]) -> float {
      if constexpr (F16) {
        float mx = 0.f;
#pragma unroll
        for (int q = 0; q < 12; ++q) mx = fmaxf(mx, fabsf(v[q]));
        float rinv;
        const float sc = pow2_scale(quad_max(mx), rinv);
        write_a_f16(A, r, u, v, sc);
        return rinv;
      } else {
        write_a_alt(A, r, u, v);
        return 1.f;
      }
    };
    // per-slot row state in shared memory: ||r||^2, ||x||, atoms taken (bit 8:
    // the row has stopped), the inverse scale of the staged operand
    auto st_rn2 = [&](int t) { return reinterpret_cast<float*>(smem + p.off_row[t]); };
    auto st_xn = [&](int t) { return reinterpret_cast<float*>(smem + p.off_row[t]) + TILE_M; };
    auto st_tc = [&](int t) { return reinterpret_cast<int*>(smem + p.off_row[t]) + 2 * TILE_M; };
    auto st_inv = [&](int t) { return reinterpret_cast<float*>(smem + p.off_row[t]) + 3 * TILE_M; };
    // row r of tile `tl` (slot t) into the staging area; its ||x||^2
    auto stage_x = [&](int t, long long tl, int r) -> float {
      const int64_t tg0 = tl * TILE_M;
      const bool tin = r < rows_of(tl);
      const float* txr = a.X + (tg0 + r) * DLSH_D;
      float x[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) x[q] = (tin && alt_dim(u, q) < DLSH_D) ? __ldg(txr + alt_dim(u, q)) : 0.f;
      float part = 0.f;
#pragma unroll
      for (int q = 0; q < 12; ++q) part = fmaf(x[q], x[q], part);
      if constexpr (XC) {
        float* xs = reinterpret_cast<float*>(smem + p.off_x[t]);
#pragma unroll
        for (int q = 0; q < 12; ++q) xs[q * 4 * TILE_M + r * 4 + u] = x[q];
      }
      st_inv(t)[r] = stage_row(r, x);
      return quad_sum(part);
    };
    // -------- the first round's signals: slot 0, then (once its copy is done) slot 1, ..
#pragma unroll 1
    for (int t = 0; t < NSL; ++t) {
      if (rounds_of(t) > 0 && ok) {
        if (!wait_staging(job_index(t, 0, 0))) ok = false;
        if (ok)
          for (int ps = 0; ps < 2; ++ps) {
            const int r = row_of(ps);
            st_rn2(t)[r] = stage_x(t, tile_of(t, 0), r);
          }
        fence_proxy_async_smem();
        if (named_bar_or(1, SVT, !ok)) ok = false;
        if (ok && vt == 0) mbar_arrive(&bar_a[t]);
      }
    }
    for (int k = 0; k < Kt[0] && ok; ++k) {
      const int nk = slots_in(k);
      for (int t = 0; t < nk; ++t) {
        const int rows = rows_of(tile_of(t, k));
        for (int ps = 0; ps < 2; ++ps) {
          const int r = row_of(ps);
          st_xn(t)[r] = sqrtf(st_rn2(t)[r]);
          st_tc(t)[r] = r < rows ? 0 : 0x100;
        }
      }
      for (int it = 0; it < s && ok; ++it) {
#pragma unroll 1
        for (int t = 0; t < nk; ++t) {
          const long long T0 = prof_on ? clock64() : 0;
          if (!mbar_wait(&cand_full[t], (fpar >> t) & 1u, a.budget)) {
            flag_status(a.status, ST_TIMEOUT);
            ok = false;
            break;
          }
          fpar ^= 1u << t;
          if (prof_on) pcs[5] += clock64() - T0;
          // both passes' candidates into registers, then release the area
          float cva[2][2];
          int cja[2][2];
          {
            const float* cv = reinterpret_cast<const float*>(smem + p.off_cand[t]);
            const int* cj = reinterpret_cast<const int*>(smem + p.off_cand[t] + TILE_M * 2 * 4);
#pragma unroll
            for (int ps = 0; ps < 2; ++ps)
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                cva[ps][hh] = cv[row_of(ps) * 2 + hh];
                cja[ps][hh] = cj[row_of(ps) * 2 + hh];
              }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&cand_empty[t]);
          float* Ls = reinterpret_cast<float*>(smem + p.off_L[t]);
          int* sel = reinterpret_cast<int*>(smem + p.off_sel[t]);
          float* ys = reinterpret_cast<float*>(smem + p.off_y[t]);
          const long long tl = tile_of(t, k);
          const int64_t g0 = tl * TILE_M;
          const int rows = rows_of(tl);
#pragma unroll 1
          for (int ps = 0; ps < 2; ++ps) {
            const int R2 = row_of(ps);
#define LS(rr, cc2) Ls[(((rr) * ((rr) + 1)) / 2 + (cc2)) * TILE_M + R2]
#define IDG(rr) LS(rr, rr)
            const bool in_tile = R2 < rows;
            const float* xr = a.X + (g0 + R2) * DLSH_D;
            // this pass's two candidates (selects, not a run-time register index)
            const float pv0 = ps ? cva[1][0] : cva[0][0], pv1 = ps ? cva[1][1] : cva[0][1];
            const int pj0 = ps ? cja[1][0] : cja[0][0], pj1 = ps ? cja[1][1] : cja[0][1];
            float rn2c = st_rn2(t)[R2];
            const float xnc = st_xn(t)[R2];
            const int stc = st_tc(t)[R2];
            const float inv_sc = st_inv(t)[R2];
            int tcc = stc & 0xff;
            bool act = (stc & 0x100) == 0 && rn2c > eps2;
            if (act) {
              // the step for a support of T atoms, compiled once per T
              auto step = [&](auto tag) {
                constexpr int T = decltype(tag)::value;
                constexpr int TA = T > 0 ? T : 1;
                float x[12], r[12];
                if constexpr (XC) {
                  const float* xs = reinterpret_cast<const float*>(smem + p.off_x[t]);
#pragma unroll
                  for (int q = 0; q < 12; ++q) x[q] = xs[q * 4 * TILE_M + R2 * 4 + u];
                } else {
#pragma unroll
                  for (int q = 0; q < 12; ++q)
                    x[q] = (in_tile && alt_dim(u, q) < DLSH_D) ? __ldg(xr + alt_dim(u, q)) : 0.f;
                }
                int sl[TA];
#pragma unroll
                for (int m = 0; m < T; ++m) sl[m] = sel[m * TILE_M + R2];
                int js = -1;
                float bestv = -1.f;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                  const float v = hh ? pv1 : pv0;
                  const int j = hh ? pj1 : pj0;
                  if (j < K && (v > bestv || (v == bestv && j < js))) {
                    bestv = v;
                    js = j;
                  }
                }
                bool dup = false;
#pragma unroll
                for (int m = 0; m < T; ++m) dup |= sl[m] == js;
                if (dup) js = -1;
                if (js < 0 || !(bestv * inv_sc > CORR_STOP_REL * xnc)) {
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
                    st_inv(t)[R2] = stage_row(R2, r);
                  else
                    ok = false;
                  if (prof_on) pcs[3] += clock64() - W5;
                }
              };
              if (tcc < 8)
                with_t<8>(tcc, step);
              else
                act = false;
            }
            st_rn2(t)[R2] = rn2c;
            st_tc(t)[R2] = tcc | (act ? 0 : 0x100);
            // last iteration: this row's codes, then its next tile's signals
            if (it + 1 == s) {
              if (in_tile) {
                const int64_t gi = g0 + R2;
                for (int mm = u; mm < s; mm += 4) {
                  a.idx[gi * s + mm] = mm < tcc ? static_cast<uint16_t>(sel[mm * TILE_M + R2]) : static_cast<uint16_t>(0);
                  if (mm >= tcc) a.coef[gi * s + mm] = 0.f;
                }
                if (u == 0) {
                  a.nnz[gi] = static_cast<uint8_t>(tcc);
                  if (a.resid_sq) a.resid_sq[gi] = rn2c;
                }
              }
              if (k + 1 < rounds_of(t) && ok) {
                if (wait_staging(job_index(t, k + 1, 0)))
                  st_rn2(t)[R2] = stage_x(t, tile_of(t, k + 1), R2);
                else
                  ok = false;
              }
            }
#undef LS
#undef IDG
          }
          fence_proxy_async_smem();
          if (named_bar_or(1, SVT, !ok)) {
            ok = false;
            break;
          }
          const bool more = it + 1 < s || k + 1 < rounds_of(t);
          if (more && vt == 0) mbar_arrive(&bar_a[t]);
          if (prof_on) {
            pcs[2] += clock64() - T0;
            pcs[4] += 1;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (prof_any && tid == 0) {
    for (int q = 0; q < 11; ++q) atomicAdd(a.prof + q, pcs[q]);
    if (blockIdx.x == 0) a.prof[11] = F16 ? (NSL == 3 ? 6 : 5) : 4;  // the variant that ran
  }
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}
