// Host side of the encoder: plans, dictionary preparation (prep_kernel,
// gram_kernel), the correlation-only kernel, kernel choice, the C ABI entry
// points, the autotuner and the multi-scene call.  The encoder kernels are in
// encode_core.cuh.
#include "encode_core.cuh"

namespace dlsh {
namespace enc {

// ---------------------------------------------------------------------------
// Dictionary preparation: padded FP32 copy, FP8 scales and the packed operand
// image, one block of 64 threads per (padded) atom.
// ---------------------------------------------------------------------------
__global__ void prep_kernel(const float* __restrict__ D, int K, int Kp, int BN, int prec,
                            float* __restrict__ D32p, uint8_t* __restrict__ img,
                            float* __restrict__ sigma, uint32_t chunk_bytes) {
  const int j = blockIdx.x;
  const int k = threadIdx.x;
  const float v = (j < K && k < DLSH_D) ? D[static_cast<size_t>(j) * DLSH_D + k] : 0.f;
  if (k < DPAD) D32p[static_cast<size_t>(j) * DPAD + k] = v;
  __shared__ float red[64];
  red[k] = fabsf(v);
  __syncthreads();
  for (int w = 32; w > 0; w >>= 1) {
    if (k < w) red[k] = fmaxf(red[k], red[k + w]);
    __syncthreads();
  }
  const float sj = red[0] > 0.f ? red[0] / FP8_MAX : 1.f;
  if (k == 0 && sigma) sigma[j] = sj;
  const int c = j / BN, n = j % BN;
  uint8_t* base = img + static_cast<size_t>(c) * chunk_bytes;
  if (prec == 1) {
    if (k < DPAD) {
      const int kb = k / 8;
      *reinterpret_cast<__nv_bfloat16*>(base + kb * BN * 16 + n * 16 + (k % 8) * 2) =
          __float2bfloat16_rn(v);
    }
  } else if (prec == 0) {
    if (k < DPAD) {
      const float hi = to_tf32(v);
      const float lo = to_tf32(v - hi);
      const int kb = k / 4;
      const uint32_t o = kb * BN * 16 + n * 16 + (k % 4) * 4;
      *reinterpret_cast<float*>(base + o) = hi;
      *reinterpret_cast<float*>(base + BN * 12 * 16 + o) = lo;
    }
  } else if (prec == OPF16X2) {
    // FP32 as two FP16 parts of 256 * v (the scale keeps the low part normal
    // down to |v| of about 2^-11; unit-norm atoms stay far below FP16's range)
    if (k < DPAD) {
      const float sv = 256.f * v;
      const __half hi = __float2half_rn(sv);
      const __half lo = __float2half_rn(sv - __half2float(hi));
      const int kb = k / 8;
      const uint32_t o = kb * BN * 16 + n * 16 + (k % 8) * 2;
      *reinterpret_cast<__half*>(base + o) = hi;
      *reinterpret_cast<__half*>(base + BN * 6 * 16 + o) = lo;
    }
  } else {
    const int kb = k / 16;
    const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(v / sj, __NV_SATFINITE, __NV_E4M3);
    base[kb * BN * 16 + n * 16 + (k % 16)] = q;
  }
}

// G = D D^T (FP32), 32 x 32 output tiles.
__global__ void gram_kernel(const float* __restrict__ D32p, int K, float* __restrict__ G) {
  __shared__ float ta[32][DPAD + 1];
  __shared__ float tb[32][DPAD + 1];
  const int j0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int f = ty * 32 + tx; f < 32 * DPAD; f += 256) {
    const int r = f / DPAD, c = f % DPAD;
    ta[r][c] = (j0 + r < K) ? D32p[static_cast<size_t>(j0 + r) * DPAD + c] : 0.f;
    tb[r][c] = (k0 + r < K) ? D32p[static_cast<size_t>(k0 + r) * DPAD + c] : 0.f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < DLSH_D; ++c) acc = fmaf(ta[r][c], tb[tx][c], acc);
    if (j0 + r < K && k0 + tx < K) G[static_cast<size_t>(j0 + r) * K + k0 + tx] = acc;
  }
}


// ---------------------------------------------------------------------------
// Correlation only: C = R D^T through the same operand packing and MMAs.
// 128 threads; thread 0 drives TMA and MMA, all threads drain TMEM.
// ---------------------------------------------------------------------------
template <int PREC, int BN>
__global__ void __launch_bounds__(128, 1)
    correlate_kernel(const float* __restrict__ R, int64_t M, int K, const uint8_t* __restrict__ img,
                     const float* __restrict__ sigma, int nchunks, uint32_t chunk_bytes,
                     uint32_t a_bytes, float* __restrict__ C, uint32_t* status, long long budget) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  uint8_t* A = smem;
  uint8_t* Bs = smem + ((a_bytes + 1023u) & ~1023u);
  // The operand regions are followed by at least 64 KB of slack so that every
  // descriptor-addressed read stays inside this CTA's shared memory.
  uint8_t* tail = Bs + ((chunk_bytes + 1023u) & ~1023u) + 65536;
  uint64_t* bar_d = reinterpret_cast<uint64_t*>(tail);
  uint64_t* bar_m = bar_d + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_m + 1);
  float* rho_s = reinterpret_cast<float*>(tail + 64);
  if (tid == 0) {
    mbar_init(bar_d, 1);
    mbar_init(bar_m, 1);
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
  const uint32_t trow = tmem_base + (static_cast<uint32_t>(warp * 32) << 16);
  uint32_t ph_d = 0, ph_m = 0;
  bool ok = true;
  const int ntiles = static_cast<int>((M + TILE_M - 1) / TILE_M);
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int64_t g = static_cast<int64_t>(tile) * TILE_M + tid;
    float r[48];
#pragma unroll
    for (int k = 0; k < 48; ++k) r[k] = (g < M && k < DLSH_D) ? R[g * DLSH_D + k] : 0.f;
    rho_s[tid] = write_a_row<PREC>(A, tid, r);
    fence_proxy_async_smem();
    __syncthreads();
    for (int c = 0; c < nchunks && ok; ++c) {
      if (tid == 0) {
        mbar_arrive_expect_tx(bar_d, chunk_bytes);
        bulk_g2s(Bs, img + static_cast<size_t>(c) * chunk_bytes, chunk_bytes, bar_d);
        if (mbar_wait(bar_d, ph_d, budget)) {
          tc_fence_after();
          issue_chunk<PREC, BN>(tmem_base, smem_u32(A), smem_u32(Bs));
          tc_commit(bar_m);
        } else {
          flag_status(status, ST_TIMEOUT);
        }
      }
      ph_d ^= 1u;
      if (!mbar_wait(bar_m, ph_m, budget)) {
        flag_status(status, ST_TIMEOUT);
        ok = false;
      }
      ph_m ^= 1u;
      tc_fence_after();
      if (ok) {
        for (int cb = 0; cb < BN; cb += 32) {
          float v[32];
          __syncwarp();
          tmem_ld32(trow + static_cast<uint32_t>(cb), v);
          if (g < M) {
#pragma unroll
            for (int k = 0; k < 32; ++k) {
              const int j = c * BN + cb + k;
              float val = v[k];
              if constexpr (PREC == 2) val *= rho_s[tid] * __ldg(sigma + j);
              if (j < K) C[g * K + j] = val;
            }
          }
        }
      }
      tc_fence_before();
      __syncthreads();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
struct Ws {
  uint32_t* status;
  float* D32p;
  float* G;
  uint8_t* img;
  float* sigma;
};

static size_t carve(void* base, const Plan& p, Ws& w) {
  Carver c(base);
  w.status = c.take<uint32_t>(64);
  w.D32p = c.take<float>(static_cast<size_t>(p.Kp) * DPAD);
  w.G = c.take<float>(static_cast<size_t>(p.K) * p.K);
  w.img = c.take<uint8_t>(static_cast<size_t>(p.nchunks) * p.chunk_bytes);
  w.sigma = c.take<float>(p.Kp);
  return c.size();
}

static int validate(const char* call, const float* D, int K, int d, int s, int prec) {
  if (d != DLSH_D) return set_error(DLSH_ERR_UNSUPPORTED, "%s: d must be 45, got %d", call, d);
  if (K < 1 || K > DLSH_MAX_K)
    return set_error(DLSH_ERR_UNSUPPORTED, "%s: K must be in [1, 65535], got %d", call, K);
  if (s < 1 || s > 16)
    return set_error(DLSH_ERR_UNSUPPORTED, "%s: s must be in [1, 16], got %d", call, s);
  if (prec < 0 || prec > 4)
    return set_error(DLSH_ERR_INVALID_ARG, "%s: unknown precision %d", call, prec);
  if (!D) return set_error(DLSH_ERR_INVALID_ARG, "%s: D is NULL", call);
  return DLSH_OK;
}
// The workspace fields (padded dictionary, Gram, operand image in 64-atom
// chunks) of the two-tile kernel, in the single-tile plan's form.
static void pair_prep_plan(const PairPlan& pp, Plan& p) {
  p = Plan{};
  p.prec = pp.prec;
  p.top4 = pp.top4;
  p.ib = pp.ib;
  p.BN = PBN;
  p.K = pp.K;
  p.Kp = pp.Kp;
  p.nchunks = pp.nchunks;
  p.s = pp.s;
  p.chunk_bytes = pp.chunk_bytes;
  p.a_bytes = pp.a_bytes;
}

template <int PREC, int BN>
static int launch_correlate(const float* R, int64_t M, const Plan& p, const Ws& w, float* C,
                            int grid, cudaStream_t st) {
  auto fn = correlate_kernel<PREC, BN>;
  uint32_t smem = ((p.a_bytes + 1023u) & ~1023u) + ((p.chunk_bytes + 1023u) & ~1023u) + 65536 +
                  64 + TILE_M * 4;
  if (smem < 120 * 1024) smem = 120 * 1024;  // one CTA per SM (whole-TMEM allocation)
  DLSH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT),
                "dlsh_correlate: cudaFuncSetAttribute");
  fn<<<grid, 128, smem, st>>>(R, M, p.K, w.img, w.sigma, p.nchunks, p.chunk_bytes, p.a_bytes, C,
                               w.status, kWaitBudget);
  count_launches(1);
  return check_launch("dlsh_correlate: launch");
}

// Launches the dictionary preparation (padded copy, Gram, operand image).
static int prepare(const float* D, const Plan& p, const Ws& w, bool gram, cudaStream_t st) {
  DLSH_CUDA_TRY(cudaMemsetAsync(w.status, 0, sizeof(uint32_t), st), "dlsh: status reset");
  prep_kernel<<<p.Kp, 64, 0, st>>>(D, p.K, p.Kp, p.BN, p.prec, w.D32p, w.img, w.sigma,
                                   p.chunk_bytes);
  count_launches(1);
  int rc = check_launch("dlsh: prep_kernel");
  if (rc) return rc;
  if (gram) {
    dim3 g((p.K + 31) / 32, (p.K + 31) / 32);
    gram_kernel<<<g, dim3(32, 8), 0, st>>>(w.D32p, p.K, w.G);
    count_launches(1);
    rc = check_launch("dlsh: gram_kernel");
  }
  return rc;
}

}  // namespace enc

// At most `cap` stages in a plan's dictionary ring (cap 0: as many as fit; a
// cap below the kernel's minimum or above the fit changes nothing).  The shared
// memory stays above half of an SM's, so that each SM holds one CTA and its
// whole tensor memory.
template <class P>
static void cap_ring(P& p, int cap, int min_stages) {
  if (cap < min_stages || cap >= p.stages) return;
  p.stages = cap;
  p.smem = p.off_ring + static_cast<uint32_t>(cap) * p.chunk_bytes;
  if (p.smem < 120 * 1024) p.smem = 120 * 1024;
}
static void cap_ring(enc::Plan& p, int cap) {
  cap_ring(p, cap, 2);
  p.resident = p.stages >= p.nchunks;
}

// The built-in encoder choice among the kernels whose plans fit: 5 (FP32 on
// selection and solver warps, FP16 parts), else 7 (FP32, one tile, FP16
// parts), else 3 (FP32, two tiles in turn), else 2 (BF16/FP8 on two warp
// groups), else 0 (one tile; the chunk width from choose_bn).
static int default_variant(bool split16_ok, bool alt_ok, bool pair_lowp_ok, bool one16_ok) {
  return split16_ok ? 5 : (one16_ok ? 7 : (alt_ok ? 3 : (pair_lowp_ok ? 2 : 0)));
}

// Entry points shared with the learning loop (learn.cu).
int encode_enqueue(const float* D, int K, const float* X, int64_t N, int s, float eps, int prec,
                   uint16_t* idx, float* coef, uint8_t* nnz, float* resid_sq, void* ws,
                   cudaStream_t st, uint32_t** status_out, unsigned long long* prof,
                   const long long* n_dev, int bn) {
  using namespace enc;
  // kernel variant (s <= 8): 2 = two tiles in flight on two warp groups,
  // 3 = two tiles served in turn by all warps (FP32), 4 / 5 = two tiles with
  // the warps split into selection and solver groups (FP32 as three TF32 / three
  // FP16 products), 6 = the same with three tiles and FP16 products, 7 = one
  // tile with FP16 products (128-atom chunks); 64 / 128 = one tile with that
  // atom-chunk width; 0 = the tuned choice, else the default below.  Bits
  // 8-15 of bn (or of the tuned choice) cap the dictionary ring's stages.
  int choice = bn != 0 ? bn : tuned_choice(K, s, prec);
  const int cap = (choice >> 8) & 255;
  choice &= 255;
  PairPlan pp;
  AltPlan ap;
  SplitPlan sp, sp16, sp16x3;
  const bool pair_ok = !prof && make_pair_plan(K, s, prec, pp) == DLSH_OK;
  const bool alt_ok = make_alt_plan(K, s, prec, ap) == DLSH_OK;
  const bool split_ok = make_split_plan(K, s, prec, sp, false) == DLSH_OK;
  const bool split16_ok = make_split_plan(K, s, prec, sp16, true) == DLSH_OK;
  const bool split16x3_ok = make_split_plan(K, s, prec, sp16x3, true, 3) == DLSH_OK;
  Plan p16;
  const bool one16_ok = prec == 0 && make_plan(K, s, prec, p16, 128, SMEM_LIMIT, true) == DLSH_OK;
  // default (measured at N = 3M, K = 1024): BF16/FP8, bound by selection and
  // solver, on two warp groups (1.2-1.3x faster than one tile); FP32 on
  // selection and solver warps with three FP16 products (1.9x faster than one
  // tile at s = 8)
  if (choice == 0) choice = default_variant(split16_ok, alt_ok, pair_ok && pp.prec != 0, one16_ok);
  if (choice == 2 && !pair_ok) choice = 0;
  if (choice == 3 && !alt_ok) choice = 0;
  if (choice == 4 && !split_ok) choice = 0;
  if (choice == 5 && !split16_ok) choice = 0;
  if (choice == 6 && !split16x3_ok) choice = 0;
  if (choice == 7 && !one16_ok) choice = 0;
  cap_ring(pp, cap, 3);
  cap_ring(ap, cap, 2);
  cap_ring(sp, cap, 2);
  cap_ring(sp16, cap, 2);
  cap_ring(sp16x3, cap, 2);
  if (choice >= 3 && choice <= 6) {
    Plan p;  // the one-tile encoder's 128-atom FP32 operand image
    if (make_plan(K, s, prec, p, 128) != DLSH_OK || p.BN != 128)
      return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode: K=%d s=%d does not fit", K, s);
    Ws w;
    carve(ws, p, w);
    if (status_out) *status_out = w.status;
    Plan pi = p;  // the operand image: TF32 hi / lo, or FP16 hi / lo (half the bytes)
    if (choice == 5 || choice == 6) {
      pi.prec = OPF16X2;
      pi.chunk_bytes = sp16.chunk_bytes;
    }
    int rc = prepare(D, pi, w, true, st);
    if (rc) return rc;
    if (N == 0 && !n_dev) return DLSH_OK;
    auto fill = [&](auto& a) {
      a.X = X;
      a.N = N;
      a.D32p = w.D32p;
      a.G = w.G;
      a.img = w.img;
      a.idx = idx;
      a.coef = coef;
      a.nnz = nnz;
      a.resid_sq = resid_sq;
      a.eps = eps;
      a.status = w.status;
      a.budget = kWaitBudget;
      a.n_dev = n_dev;
      a.prof = prof;
    };
    const int ntiles = static_cast<int>((N + TILE_M - 1) / TILE_M);
    int sms = device_sm_count();
    if (sms <= 0) sms = 1;
    // two (three) tiles per CTA: enough CTAs for every SM, fewer when the
    // tiles run out (a count read on the device takes every SM)
    const int per = choice == 6 ? 3 : 2;
    const int want = (ntiles + per - 1) / per;
    const int grid = (!n_dev && want < sms) ? (want > 0 ? want : 1) : sms;
    if (choice >= 4) {
      SplitArgs a{};
      fill(a);
      a.p = choice == 6 ? sp16x3 : (choice == 5 ? sp16 : sp);
      if (choice == 6) return launch_split<true, 3>(a, grid, st);
      return choice == 5 ? launch_split<true, 2>(a, grid, st) : launch_split<false, 2>(a, grid, st);
    }
    AltArgs a{};
    fill(a);
    a.p = ap;
    return launch_alt(a, grid, st);
  }
  if (choice == 2) {
    Plan p;
    pair_prep_plan(pp, p);
    Ws w;
    carve(ws, p, w);
    if (status_out) *status_out = w.status;
    int rc = prepare(D, p, w, true, st);
    if (rc) return rc;
    if (N == 0 && !n_dev) return DLSH_OK;
    PairArgs a{};
    a.X = X;
    a.N = N;
    a.D32p = w.D32p;
    a.G = w.G;
    a.img = w.img;
    a.sigma = w.sigma;
    a.idx = idx;
    a.coef = coef;
    a.nnz = nnz;
    a.resid_sq = resid_sq;
    a.eps = eps;
    a.status = w.status;
    a.budget = kWaitBudget;
    a.n_dev = n_dev;
    a.p = pp;
    const int ntiles = static_cast<int>((N + TILE_M - 1) / TILE_M);
    int sms = device_sm_count();
    if (sms <= 0) sms = 1;
    // two tiles per CTA: enough CTAs for every SM, fewer when the tiles run out
    // (a count read on the device takes every SM)
    const int grid = (!n_dev && (ntiles + 1) / 2 < sms) ? ((ntiles + 1) / 2 > 0 ? (ntiles + 1) / 2 : 1) : sms;
    if (pp.prec == 0) return launch_pair<0, false>(a, grid, st);
    if (pp.prec == 1) return pp.top4 ? launch_pair<1, true>(a, grid, st) : launch_pair<1, false>(a, grid, st);
    return pp.top4 ? launch_pair<2, true>(a, grid, st) : launch_pair<2, false>(a, grid, st);
  }
  Plan p;
  if (make_plan(K, s, prec, p, (choice >= 2 && choice <= 7) ? 0 : choice, SMEM_LIMIT, choice == 7) != DLSH_OK)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode: K=%d s=%d precision=%d does not fit", K,
                     s, prec);
  cap_ring(p, cap);
  Ws w;
  carve(ws, p, w);
  if (status_out) *status_out = w.status;
  int rc = prepare(D, p, w, true, st);
  if (rc) return rc;
  if (N == 0 && !n_dev) return DLSH_OK;
  Args a{};  // value-initialised: no scene table, no device-side count, no profiling
  a.X = X;
  a.N = N;
  a.D32p = w.D32p;
  a.G = w.G;
  a.img = w.img;
  a.sigma = w.sigma;
  a.idx = idx;
  a.coef = coef;
  a.nnz = nnz;
  a.resid_sq = resid_sq;
  a.eps = eps;
  a.status = w.status;
  a.budget = kWaitBudget;
  a.prof = prof;
  a.n_dev = n_dev;
  a.p = p;
  const int ntiles = static_cast<int>((N + TILE_M - 1) / TILE_M);
  int sms = device_sm_count();
  if (sms <= 0) sms = 1;
  const int grid = (n_dev || ntiles > sms) ? sms : (ntiles > 0 ? ntiles : 1);
  if (p.BN == 128) {
    if (p.prec == 0) return launch_encode<0, 128>(a, grid, st);
    if (p.prec == OPF16X2) return launch_encode<OPF16X2, 128>(a, grid, st);
    if (p.prec == 1)
      return p.top4 ? launch_encode<1, 128, true>(a, grid, st) : launch_encode<1, 128>(a, grid, st);
    return p.top4 ? launch_encode<2, 128, true>(a, grid, st) : launch_encode<2, 128>(a, grid, st);
  }
  return launch_encode<0, 64>(a, grid, st);
}

// Prepares the dictionary (padded FP32 copy, Gram, operand image) in an
// encoder workspace and returns pointers into it.
int encode_prepare_only(const float* D, int K, int s, int prec, void* ws, cudaStream_t st,
                        const float** D32p, const float** G, uint32_t** status) {
  using namespace enc;
  Plan p;
  if (make_plan(K, s, prec, p) != DLSH_OK)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh: K=%d s=%d does not fit", K, s);
  Ws w;
  carve(ws, p, w);
  *D32p = w.D32p;
  *G = w.G;
  *status = w.status;
  return prepare(D, p, w, true, st);
}

// Largest workspace over the chunk widths the plan may pick.
size_t encode_ws_bytes(int K, int s, int prec) {
  size_t best = 0;
  for (int bn : {64, 128, -128}) {  // -128: 128-atom chunks with FP16 parts
    enc::Plan p;
    if (enc::make_plan(K, s, prec, p, bn < 0 ? -bn : bn, enc::SMEM_LIMIT, bn < 0) != DLSH_OK) continue;
    enc::Ws w;
    const size_t b = enc::carve(nullptr, p, w);
    if (b > best) best = b;
  }
  enc::PairPlan pp;
  if (best > 0 && enc::make_pair_plan(K, s, prec, pp) == DLSH_OK) {
    enc::Plan p;
    enc::pair_prep_plan(pp, p);
    enc::Ws w;
    const size_t b = enc::carve(nullptr, p, w);
    if (b > best) best = b;
  }
  return best;
}

}  // namespace dlsh

extern "C" {

size_t dlsh_encode_workspace_size(int K, int d, int s, int precision) {
  if (d != DLSH_D || K < 1 || K > DLSH_MAX_K || s < 1 || s > 16 || precision < 0 || precision > 4)
    return 0;
  return dlsh::encode_ws_bytes(K, s, precision);
}

int dlsh_encode_variant(int K, int s, int precision) {
  using namespace dlsh::enc;
  if (K < 1 || K > DLSH_MAX_K || s < 1 || s > 16 || precision < 0 || precision > 4) return 0;
  PairPlan pp;
  AltPlan ap;
  SplitPlan sp16;
  Plan p;
  const bool pair_ok = make_pair_plan(K, s, precision, pp) == DLSH_OK;
  const bool alt_ok = make_alt_plan(K, s, precision, ap) == DLSH_OK;
  const bool split16_ok = make_split_plan(K, s, precision, sp16, true) == DLSH_OK;
  Plan p16;
  const bool one16_ok = precision == 0 && make_plan(K, s, precision, p16, 128, SMEM_LIMIT, true) == DLSH_OK;
  const int v = dlsh::default_variant(split16_ok, alt_ok, pair_ok && pp.prec != 0, one16_ok);
  if (v != 0) return v;
  return make_plan(K, s, precision, p, 0) == DLSH_OK ? 1 : 0;
}

int dlsh_encode(const float* D, int K, int d, const float* X, int64_t N, int s, float eps,
                int precision, uint16_t* idx, float* coef, uint8_t* nnz, float* resid_sq,
                void* ws, size_t ws_bytes, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  int rc = enc::validate("dlsh_encode", D, K, d, s, precision);
  if (rc) return rc;
  if (N < 0) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode: N < 0");
  if (N > 0 && (!X || !idx || !coef || !nnz))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode: NULL X/idx/coef/nnz");
  if (!(eps >= 0.f)) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode: eps must be >= 0");
  const size_t need = encode_ws_bytes(K, s, precision);
  if (need == 0)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode: K=%d s=%d precision=%d does not fit", K,
                     s, precision);
  rc = check_workspace(ws, ws_bytes, need, "dlsh_encode");
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* status = nullptr;
  rc = encode_enqueue(D, K, X, N, s, eps, precision, idx, coef, nnz, resid_sq, ws, st, &status,
                      nullptr, nullptr);
  if (rc) return rc;
  return finish(st, status, flags, "dlsh_encode");
}

int dlsh_encode_profile(const float* D, int K, int d, const float* X, int64_t N, int s, float eps,
                        int precision, uint16_t* idx, float* coef, uint8_t* nnz, float* resid_sq,
                        void* ws, size_t ws_bytes, unsigned long long* cycles, void* stream,
                        int flags) {
  using namespace dlsh;
  clear_error();
  int rc = enc::validate("dlsh_encode_profile", D, K, d, s, precision);
  if (rc) return rc;
  if (N < 0 || (N > 0 && (!X || !idx || !coef || !nnz)) || !cycles)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_profile: bad arguments");
  rc = check_workspace(ws, ws_bytes, encode_ws_bytes(K, s, precision), "dlsh_encode_profile");
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DLSH_CUDA_TRY(cudaMemsetAsync(cycles, 0, 12 * sizeof(unsigned long long), st),
                "dlsh_encode_profile: reset");
  uint32_t* status = nullptr;
  rc = encode_enqueue(D, K, X, N, s, eps, precision, idx, coef, nnz, resid_sq, ws, st, &status,
                      cycles, nullptr);
  if (rc) return rc;
  return finish(st, status, flags, "dlsh_encode_profile");
}

int dlsh_correlate(const float* D, int K, int d, const float* R, int64_t M, int precision,
                   float* C, void* ws, size_t ws_bytes, void* stream, int flags) {
  using namespace dlsh;
  using namespace dlsh::enc;
  clear_error();
  int rc = validate("dlsh_correlate", D, K, d, 1, precision);
  if (rc) return rc;
  if (M < 0) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_correlate: M < 0");
  if (M > 0 && (!R || !C)) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_correlate: NULL R/C");
  Plan p;
  if (make_plan(K, 1, precision, p) != DLSH_OK)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_correlate: K=%d does not fit", K);
  const size_t need = encode_ws_bytes(K, 1, precision);
  rc = check_workspace(ws, ws_bytes, need, "dlsh_correlate");
  if (rc) return rc;
  Ws w;
  carve(ws, p, w);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = prepare(D, p, w, false, st);
  if (rc) return rc;
  if (M > 0) {
    const int ntiles = static_cast<int>((M + TILE_M - 1) / TILE_M);
    int sms = device_sm_count();
    if (sms <= 0) sms = 1;
    const int grid = ntiles < sms ? ntiles : sms;
    if (p.prec == 0) rc = launch_correlate<0, 128>(R, M, p, w, C, grid, st);
    else if (p.prec == 1) rc = launch_correlate<1, 128>(R, M, p, w, C, grid, st);
    else rc = launch_correlate<2, 128>(R, M, p, w, C, grid, st);
    if (rc) return rc;
  }
  return finish(st, w.status, flags, "dlsh_correlate");
}

}  // extern "C"

// ===========================================================================
// Autotuner: times the encoder at each admissible atom-chunk width on the
// caller's sample and records the fastest per (K, s, precision), in memory and,
// if DLSH_AUTOTUNE_CACHE names a file, as JSON lines there (read at first use).
// ===========================================================================
namespace dlsh {
namespace enc {

// The recorded choice for (K, s, precision): the kernel variant in the low
// byte, the ring-stage cap above it (0: none recorded).
int tuned_choice(int K, int s, int prec) {
  char key[64];
  snprintf(key, sizeof(key), "encode K=%d s=%d p=%d", K, s, prec);
  int v[2] = {0, 0};
  if (!tune_get(key, v, 2)) return 0;
  return (v[0] & 255) | ((v[1] & 255) << 8);
}

int tuned_bn(int K, int s, int prec) { return tuned_choice(K, s, prec) & 255; }

static void record_tuned(int K, int s, int prec, int choice) {
  char key[64];
  snprintf(key, sizeof(key), "encode K=%d s=%d p=%d", K, s, prec);
  const int v[2] = {choice & 255, (choice >> 8) & 255};
  tune_put(key, v, 2);
}

static void forget_tuned(int K, int s, int prec) {
  char key[64];
  snprintf(key, sizeof(key), "encode K=%d s=%d p=%d", K, s, prec);
  tune_put(key, nullptr, 0);
}

}  // namespace enc
}  // namespace dlsh

extern "C" int dlsh_tuned_encode(int K, int s, int precision) {
  if (K < 1 || K > DLSH_MAX_K || s < 1 || s > 16 || precision < 0 || precision > 4) return 0;
  return dlsh::enc::tuned_choice(K, s, precision);
}

extern "C" int dlsh_autotune_encode(const float* D, int K, int d, const float* X, int64_t N, int s,
                                    int precision, uint16_t* idx, float* coef, uint8_t* nnz,
                                    float* resid_sq, void* ws, size_t ws_bytes, void* stream,
                                    int* best_bn) {
  using namespace dlsh;
  using namespace dlsh::enc;
  clear_error();
  int rc = validate("dlsh_autotune_encode", D, K, d, s, precision);
  if (rc) return rc;
  if (N < 1 || !X || !idx || !coef || !nnz)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_autotune_encode: need a non-empty sample");
  rc = check_workspace(ws, ws_bytes, encode_ws_bytes(K, s, precision), "dlsh_autotune_encode");
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  DLSH_CUDA_TRY(cudaEventCreate(&e0), "dlsh_autotune_encode: event");
  DLSH_CUDA_TRY(cudaEventCreate(&e1), "dlsh_autotune_encode: event");
  // the time of one choice: a warm-up run, then two timed runs
  auto trial = [&](int choice, float* ms_out) -> int {
    record_tuned(K, s, precision, choice);  // force this choice for the trial runs
    uint32_t* status = nullptr;
    float ms_sum = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, st);
      const int r = encode_enqueue(D, K, X, N, s, 0.f, precision, idx, coef, nnz, resid_sq, ws, st, &status,
                                   nullptr, nullptr);
      cudaEventRecord(e1, st);
      if (r) return r;
      DLSH_CUDA_TRY(cudaEventSynchronize(e1), "dlsh_autotune_encode: event");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) ms_sum += ms;
    }
    *ms_out = ms_sum;
    return DLSH_OK;
  };
  // first the kernel variant, each with as many ring stages as fit ...
  int best = 0, best_stages = 0, min_stages = 2;
  float best_ms = 0.f;
  for (int bn : {64, 128, 2, 3, 4, 5, 6, 7}) {
    Plan p;
    PairPlan pp;
    AltPlan ap;
    SplitPlan sp;
    if (bn == 2 ? make_pair_plan(K, s, precision, pp) != DLSH_OK
                : bn == 3 ? make_alt_plan(K, s, precision, ap) != DLSH_OK
                : bn >= 4 && bn <= 6 ? make_split_plan(K, s, precision, sp, bn >= 5, bn == 6 ? 3 : 2) != DLSH_OK
                : bn == 7 ? (precision != 0 || make_plan(K, s, precision, p, 128, SMEM_LIMIT, true) != DLSH_OK)
                          : (make_plan(K, s, precision, p, bn) != DLSH_OK || p.BN != bn))
      continue;
    float ms = 0.f;
    rc = trial(bn, &ms);
    if (rc) break;
    if (best == 0 || ms < best_ms) {
      best = bn;
      best_ms = ms;
      best_stages = bn == 2 ? pp.stages : bn == 3 ? ap.stages : (bn >= 4 && bn <= 6) ? sp.stages : p.stages;
      min_stages = bn == 2 ? 3 : 2;
    }
  }
  // ... then, for the fastest, a shallower dictionary ring (half the stages,
  // and the kernel's minimum)
  if (!rc && best != 0) {
    const int v = best;
    int caps[2] = {best_stages / 2, min_stages}, ncap = 0;
    for (int c : {best_stages / 2, min_stages})
      if (c >= min_stages && c < best_stages && (ncap == 0 || caps[0] != c)) caps[ncap++] = c;
    for (int i = 0; i < ncap && !rc; ++i) {
      float ms = 0.f;
      rc = trial(v | (caps[i] << 8), &ms);
      if (!rc && ms < best_ms) {
        best = v | (caps[i] << 8);
        best_ms = ms;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    // keep no trial choice: the best one timed so far, else none
    if (best != 0) record_tuned(K, s, precision, best);
    else forget_tuned(K, s, precision);
    return rc;
  }
  if (best == 0) return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_autotune_encode: no admissible width");
  record_tuned(K, s, precision, best);
  if (best_bn) *best_bn = best;
  return finish(st, nullptr, 0, "dlsh_autotune_encode");
}

// ===========================================================================
// Multi-scene encoding.  Every scene is encoded by the single-scene encoder
// with its own plan (the chunk width and staging a dlsh_encode call of that
// scene would pick, so the codes are bitwise those of separate calls), on one
// of a few internal streams forked from the caller's stream with an event and
// joined back the same way.  Scenes are dealt to the streams in decreasing
// order of total cost (N*K*s), so small scenes fill the SMs the large ones
// leave idle.  Event record and wait are captured as graph dependencies, so
// the whole call can be captured into a CUDA graph.
// ===========================================================================
#include <mutex>

namespace dlsh {
namespace enc {

constexpr int MAX_SCENES = 32;
constexpr int kStreams = 4;
constexpr int kMaxDevices = 64;

struct StatusList {
  const uint32_t* w[MAX_SCENES];
  int n;
};

// out |= the status words of every scene.
__global__ void or_status_list_kernel(const StatusList l, uint32_t* out) {
  uint32_t v = 0;
  for (int i = 0; i < l.n; ++i) v |= l.w[i][0];
  if (v) atomicOr(out, v);
}

struct Fork {
  cudaStream_t s[kStreams];
  cudaEvent_t fork, join[kStreams];
  bool ready = false;
};
static std::mutex g_fork_mu;
static Fork g_fork[kMaxDevices];

// Per-scene workspace regions: one status word for the call, then a
// single-scene encoder workspace per scene.
static size_t multi_carve(void* base, const dlsh_scene* sc, int n, int prec, uint32_t** status,
                          void** per) {
  Carver c(base);
  *status = c.take<uint32_t>(64);
  for (int i = 0; i < n; ++i) per[i] = c.take<uint8_t>(encode_ws_bytes(sc[i].K, sc[i].s, prec));
  return c.size();
}

static int multi_validate(const dlsh_scene* sc, int n, int prec, int bn) {
  if (!sc || n < 1 || n > MAX_SCENES)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_multi: 1..%d scenes", MAX_SCENES);
  if (prec < 0 || prec > 4)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_multi: unknown precision %d", prec);
  const int v = bn & 255, cap = bn >> 8;
  if (bn < 0 || (v != 0 && (v < 2 || v > 7) && v != 64 && v != 128) || cap == 1 || cap > 32)
    return set_error(DLSH_ERR_INVALID_ARG,
                     "dlsh_encode_multi: bn must be 0, 2..7, 64 or 128, plus 256 x a ring cap of 2..32");
  for (int i = 0; i < n; ++i) {
    const dlsh_scene& x = sc[i];
    if (!x.D || x.K < 1 || x.K > DLSH_MAX_K || x.s < 1 || x.s > 16 || x.N < 0 || !(x.eps >= 0.f))
      return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_multi: scene %d has bad sizes", i);
    if (x.N > 0 && (!x.X || !x.idx || !x.coef || !x.nnz))
      return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_multi: scene %d has a NULL array", i);
    Plan p;
    if (make_plan(x.K, x.s, prec, p, (v >= 2 && v <= 7) ? 0 : v) != DLSH_OK)
      return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode_multi: scene %d (K=%d s=%d) does not fit",
                       i, x.K, x.s);
  }
  return DLSH_OK;
}

static int fork_streams(Fork** out) {
  int dev = 0;
  DLSH_CUDA_TRY(cudaGetDevice(&dev), "dlsh_encode_multi: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode_multi: device %d out of range", dev);
  Fork& f = g_fork[dev];
  if (!f.ready) {
    for (int i = 0; i < kStreams; ++i) {
      DLSH_CUDA_TRY(cudaStreamCreateWithFlags(&f.s[i], cudaStreamNonBlocking),
                    "dlsh_encode_multi: stream");
      DLSH_CUDA_TRY(cudaEventCreateWithFlags(&f.join[i], cudaEventDisableTiming),
                    "dlsh_encode_multi: event");
    }
    DLSH_CUDA_TRY(cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming),
                  "dlsh_encode_multi: event");
    f.ready = true;
  }
  *out = &f;
  return DLSH_OK;
}

}  // namespace enc
}  // namespace dlsh

extern "C" size_t dlsh_encode_multi_workspace_size(const dlsh_scene* scenes, int n, int precision,
                                                   int bn) {
  using namespace dlsh;
  using namespace dlsh::enc;
  if (multi_validate(scenes, n, precision, bn) != DLSH_OK) return 0;
  uint32_t* status;
  void* per[MAX_SCENES];
  return multi_carve(nullptr, scenes, n, precision, &status, per);
}

extern "C" int dlsh_encode_multi(const dlsh_scene* scenes, int n, int precision, int bn, void* ws,
                                 size_t ws_bytes, void* stream, int flags) {
  using namespace dlsh;
  using namespace dlsh::enc;
  clear_error();
  int rc = multi_validate(scenes, n, precision, bn);
  if (rc) return rc;
  uint32_t* status = nullptr;
  void* per[MAX_SCENES];
  rc = check_workspace(ws, ws_bytes, multi_carve(nullptr, scenes, n, precision, &status, per),
                       "dlsh_encode_multi");
  if (rc) return rc;
  multi_carve(ws, scenes, n, precision, &status, per);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DLSH_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(uint32_t), st), "dlsh_encode_multi: reset");
  int order[MAX_SCENES];
  int m = 0;
  for (int i = 0; i < n; ++i)
    if (scenes[i].N > 0) order[m++] = i;
  std::sort(order, order + m, [&](int a, int b) {
    const double ca = static_cast<double>(scenes[a].N) * scenes[a].K * scenes[a].s;
    const double cb = static_cast<double>(scenes[b].N) * scenes[b].K * scenes[b].s;
    return ca > cb || (ca == cb && a < b);
  });
  if (m > 0) {
    std::lock_guard<std::mutex> lock(g_fork_mu);
    Fork* f = nullptr;
    rc = fork_streams(&f);
    if (rc) return rc;
    const int used = m < kStreams ? m : kStreams;
    DLSH_CUDA_TRY(cudaEventRecord(f->fork, st), "dlsh_encode_multi: fork");
    for (int k = 0; k < used; ++k)
      DLSH_CUDA_TRY(cudaStreamWaitEvent(f->s[k], f->fork, 0), "dlsh_encode_multi: fork");
    StatusList sl{};
    sl.n = m;
    for (int q = 0; q < m; ++q) {
      const dlsh_scene& x = scenes[order[q]];
      uint32_t* sst = nullptr;
      rc = encode_enqueue(x.D, x.K, x.X, x.N, x.s, x.eps, precision, x.idx, x.coef, x.nnz,
                          x.resid_sq, per[order[q]], f->s[q % kStreams], &sst, nullptr, nullptr, bn);
      if (rc) break;
      sl.w[q] = sst;
    }
    // the join is recorded even after a failed enqueue, so that no internal
    // stream is left forked from a stream under capture
    for (int k = 0; k < used; ++k) {
      DLSH_CUDA_TRY(cudaEventRecord(f->join[k], f->s[k]), "dlsh_encode_multi: join");
      DLSH_CUDA_TRY(cudaStreamWaitEvent(st, f->join[k], 0), "dlsh_encode_multi: join");
    }
    if (rc) return rc;
    or_status_list_kernel<<<1, 1, 0, st>>>(sl, status);
    count_launches(1);
    rc = check_launch("dlsh_encode_multi: status");
    if (rc) return rc;
  }
  return finish(st, status, flags, "dlsh_encode_multi");
}
