// Learned support proposal, second half: OMP restricted to the MLP's 2s
// candidate atoms, then plain OMP (Sec. 2.1) as the fallback.
//
// restricted_omp_kernel  one lane per candidate (a signal's m candidates on m
//                        lanes of a warp).  alpha = D_C^T x once; then per step
//                        the correlations with the least-squares residual come
//                        from the lanes' projected Gram columns and y = L^-1
//                        D_I^T x, the argmax is a shuffle reduction, and adding
//                        an atom costs one Gram entry per lane.  The final
//                        residual is recomputed explicitly.
// fallback               "exact": plain OMP on every signal, keep whichever code
//                        has the smaller residual (ties keep the learned one);
//                        "deploy": plain OMP only for signals whose learned
//                        residual exceeds tau, compacted, encoded with a
//                        device-side count, and scattered back.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "host.hpp"
#include "internal.hpp"

namespace dlsh {

namespace lrn {

constexpr int RW = 8;  // warps per block of the restricted OMP
constexpr float CORR_STOP_REL = 1e-7f;
constexpr float PIVOT_MIN = 1e-6f;
constexpr int DPAD = 48;

__host__ __device__ constexpr int tri(int n) { return n * (n + 1) / 2; }

// One lane per candidate: M lanes serve one signal, 32 / M signals per warp.
// Lane q owns candidate q (atom j_q) and keeps, for the current support I,
//   v_q = L^-1 G_{I,q}   (L L^T = G_II, the Cholesky factor of the support's Gram)
// while every lane of the signal keeps y = L^-1 D_I^T x.  The correlation with
// the least-squares residual is then c_q = alpha_q - v_q . y (alpha = D_C^T x),
// the new atom p's factor row is w = v_p (taken from lane p with shuffles), and
// adding p appends (G_qp - w . v_q) / ell to v_q and (alpha_p - w . y) / ell to
// y, ell = sqrt(G_pp - w . w).  Each step is O(t) per lane; gamma comes from
// one back substitution L^T gamma = y at the end, and the reported residual is
// recomputed explicitly as x - D_I gamma.
template <int M, int SMAX>
__global__ void __launch_bounds__(RW * 32)
    restricted_omp_kernel(const float* __restrict__ X, long long N, const float* __restrict__ D32p,
                          const float* __restrict__ G, int K, const uint16_t* __restrict__ cand,
                          int s, float eps, uint16_t* __restrict__ idx, float* __restrict__ coef,
                          uint8_t* __restrict__ nnz, float* __restrict__ resid,
                          uint32_t* status) {
  constexpr int SPW = 32 / M;
  __shared__ float Lsh[RW][SPW][tri(SMAX)];  // the factor's rows, for the final solve
  __shared__ float Ish[RW][SPW][SMAX];       // 1 / L(m, m)
  __shared__ int Jsh[RW][SPW][SMAX];         // selected atoms in order
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = lane % M, g = lane / M;
  const long long n = (static_cast<long long>(blockIdx.x) * RW + warp) * SPW + g;
  const bool live = n < N;
  float* Lg = Lsh[warp][g];
  float* Ig = Ish[warp][g];
  int* Jg = Jsh[warp][g];
  int j = 0;
  bool bad = false;
  if (live) {
    j = cand[n * M + q];
    if (j >= K) {
      bad = true;
      j = 0;
    }
  }
  // alpha_q = d_q . x and ||x||^2 (every lane of a signal reads the same x)
  float alpha = 0.f, xn2 = 0.f;
  if (live) {
    const float4* dr = reinterpret_cast<const float4*>(D32p + static_cast<size_t>(j) * DPAD);
    const float* xr = X + n * DLSH_D;
#pragma unroll
    for (int u = 0; u < 12; ++u) {
      const float4 dv = __ldg(dr + u);
      // the row holds 45 values: dims 45..47 are the dictionary's zero padding
      const float x0 = __ldg(xr + 4 * u);
      const float x1 = 4 * u + 1 < DLSH_D ? __ldg(xr + 4 * u + 1) : 0.f;
      const float x2 = 4 * u + 2 < DLSH_D ? __ldg(xr + 4 * u + 2) : 0.f;
      const float x3 = 4 * u + 3 < DLSH_D ? __ldg(xr + 4 * u + 3) : 0.f;
      alpha = fmaf(dv.x, x0, alpha);
      alpha = fmaf(dv.y, x1, alpha);
      alpha = fmaf(dv.z, x2, alpha);
      alpha = fmaf(dv.w, x3, alpha);
      xn2 = fmaf(x0, x0, xn2);
      xn2 = fmaf(x1, x1, xn2);
      xn2 = fmaf(x2, x2, xn2);
      xn2 = fmaf(x3, x3, xn2);
    }
  }
  const float gself = live ? __ldg(G + static_cast<size_t>(j) * K + j) : 0.f;
  const float xnorm = sqrtf(xn2);
  float v[SMAX], y[SMAX];
#pragma unroll
  for (int m = 0; m < SMAX; ++m) v[m] = y[m] = 0.f;
  bool act = live, chosen = false;
  int t = 0;
  for (int it = 0; it < s; ++it) {
    if (act && eps > 0.f) {
      // ||r||^2 = ||x||^2 - y . y for the current least-squares fit
      float yy = 0.f;
#pragma unroll
      for (int m = 0; m < SMAX; ++m)
        if (m < t) yy = fmaf(y[m], y[m], yy);
      if (xn2 - yy <= eps * eps) act = false;
    }
    float c = alpha;
#pragma unroll
    for (int m = 0; m < SMAX; ++m)
      if (m < t) c = fmaf(-v[m], y[m], c);
    // key: |c| (a non-negative float orders as its bits), then the smaller
    // atom id, then the lane (unique); 0 = no candidate
    const float ac = fabsf(c);
    unsigned long long key = 0ull;
    if (act && !chosen && ac >= 0.f)
      key = (static_cast<unsigned long long>(__float_as_uint(ac)) << 32) |
            (static_cast<unsigned long long>(0xFFFFu - static_cast<unsigned>(j)) << 5) |
            static_cast<unsigned long long>(31 - q);
#pragma unroll
    for (int o = 1; o < M; o <<= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
      key = other > key ? other : key;
    }
    const float best = __uint_as_float(static_cast<uint32_t>(key >> 32));
    const int jp = 0xFFFF - static_cast<int>((key >> 5) & 0xFFFFu);
    const int src = g * M + 31 - static_cast<int>(key & 31u);
    if (key == 0ull || !(best > CORR_STOP_REL * xnorm)) act = false;
    // the new atom's factor row w = v_p, its Gram diagonal and alpha_p
    float w[SMAX];
#pragma unroll
    for (int m = 0; m < SMAX; ++m) w[m] = __shfl_sync(0xffffffffu, v[m], src & 31);
    const float gpp = __shfl_sync(0xffffffffu, gself, src & 31);
    const float ap = __shfl_sync(0xffffffffu, alpha, src & 31);
    if (act) {
      const float gqp = __ldg(G + static_cast<size_t>(j) * K + jp);
      float wn2 = 0.f;
#pragma unroll
      for (int m = 0; m < SMAX; ++m)
        if (m < t) wn2 = fmaf(w[m], w[m], wn2);
      const float ell2 = gpp - wn2;
      if (!(ell2 > PIVOT_MIN * gpp)) {
        act = false;
      } else {
        const float ell = sqrtf(ell2);
        const float iell = 1.f / ell;
        float vt = gqp, yt = ap;
#pragma unroll
        for (int m = 0; m < SMAX; ++m) {
          if (m < t) {
            vt = fmaf(-w[m], v[m], vt);
            yt = fmaf(-w[m], y[m], yt);
          }
        }
        vt *= iell;
        yt *= iell;
#pragma unroll
        for (int m = 0; m < SMAX; ++m) {
          if (m == t) {
            v[m] = vt;
            y[m] = yt;
          }
        }
        if (q == 0) {
#pragma unroll
          for (int m = 0; m < SMAX; ++m)
            if (m < t) Lg[tri(t) + m] = w[m];
          Lg[tri(t) + t] = ell;
          Ig[t] = iell;
          Jg[t] = jp;
        }
        chosen |= (lane == src);
        ++t;
      }
    }
  }
  __syncwarp();
  // gamma from L^T gamma = y (every lane of the signal, identical values)
  float gam[SMAX];
#pragma unroll
  for (int m = SMAX - 1; m >= 0; --m) {
    gam[m] = 0.f;
    if (m < t) {
      float acc = y[m];
#pragma unroll
      for (int r = m + 1; r < SMAX; ++r)
        if (r < t) acc = fmaf(-Lg[tri(r) + m], gam[r], acc);
      gam[m] = acc * Ig[m];
    }
  }
  // explicit residual of the final code: lane q takes dimensions q, q + M, ...
  float r2 = 0.f;
  if (live) {
    for (int k = q; k < DLSH_D; k += M) {
      float r = __ldg(X + n * DLSH_D + k);
#pragma unroll
      for (int m = 0; m < SMAX; ++m)
        if (m < t) r = fmaf(-gam[m], __ldg(D32p + static_cast<size_t>(Jg[m]) * DPAD + k), r);
      r2 = fmaf(r, r, r2);
    }
  }
#pragma unroll
  for (int o = 1; o < M; o <<= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  if (live) {
#pragma unroll
    for (int m = 0; m < SMAX; ++m) {
      if (m < s && m % M == q) {
        idx[n * s + m] = m < t ? static_cast<uint16_t>(Jg[m]) : static_cast<uint16_t>(0);
        coef[n * s + m] = m < t ? gam[m] : 0.f;
      }
    }
    if (q == 0) {
      nnz[n] = static_cast<uint8_t>(t);
      resid[n] = r2;
    }
  }
  if (bad) flag_status(status, ST_BAD_INPUT);
}

// exact mode: keep the plain code where its residual is smaller (1e-6 relative)
__global__ void choose_kernel(long long N, int s, const float* __restrict__ rL,
                              const float* __restrict__ rP, const uint16_t* __restrict__ iP,
                              const float* __restrict__ cP, const uint8_t* __restrict__ nP,
                              uint16_t* __restrict__ idx, float* __restrict__ coef,
                              uint8_t* __restrict__ nnz, float* __restrict__ resid,
                              unsigned long long* __restrict__ nfb) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  bool fb = false;
  if (i < N) {
    fb = sqrtf(rL[i]) > sqrtf(rP[i]) * (1.f + 1e-6f);
    if (fb) {
      for (int m = 0; m < s; ++m) {
        idx[i * s + m] = iP[i * s + m];
        coef[i * s + m] = cP[i * s + m];
      }
      nnz[i] = nP[i];
      resid[i] = rP[i];
    }
  }
  const unsigned cnt = __popc(__ballot_sync(0xffffffffu, fb));
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(nfb, static_cast<unsigned long long>(cnt));
}

// deploy mode: flags, per-block counts, offsets, compaction (signal order)
constexpr int CB = 1024;
__global__ void fb_count_kernel(const float* __restrict__ rL, long long N, float tau2,
                                int* __restrict__ part) {
  __shared__ int red[CB];
  const long long i = static_cast<long long>(blockIdx.x) * CB + threadIdx.x;
  red[threadIdx.x] = (i < N && rL[i] > tau2) ? 1 : 0;
  __syncthreads();
  for (int w = CB / 2; w > 0; w >>= 1) {
    if (static_cast<int>(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void fb_scan_kernel(int* part, int nblocks, long long* total) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    long long run = 0;
    for (int b = 0; b < nblocks; ++b) {
      const int v = part[b];
      part[b] = static_cast<int>(run);
      run += v;
    }
    *total = run;
  }
}
__global__ void fb_compact_kernel(const float* __restrict__ rL, const float* __restrict__ X,
                                  long long N, float tau2, const int* __restrict__ part,
                                  long long* __restrict__ list, float* __restrict__ Xfb) {
  __shared__ int sc[CB];
  const long long i = static_cast<long long>(blockIdx.x) * CB + threadIdx.x;
  const int f = (i < N && rL[i] > tau2) ? 1 : 0;
  sc[threadIdx.x] = f;
  __syncthreads();
  for (int o = 1; o < CB; o <<= 1) {
    const int v = static_cast<int>(threadIdx.x) >= o ? sc[threadIdx.x - o] : 0;
    __syncthreads();
    sc[threadIdx.x] += v;
    __syncthreads();
  }
  if (f) {
    const long long pos = part[blockIdx.x] + sc[threadIdx.x] - 1;
    list[pos] = i;
    for (int k = 0; k < DLSH_D; ++k) Xfb[pos * DLSH_D + k] = X[i * DLSH_D + k];
  }
}
__global__ void fb_scatter_kernel(const long long* __restrict__ list, const long long* __restrict__ total,
                                  int s, const uint16_t* __restrict__ iF, const float* __restrict__ cF,
                                  const uint8_t* __restrict__ nF, const float* __restrict__ rF,
                                  uint16_t* __restrict__ idx, float* __restrict__ coef,
                                  uint8_t* __restrict__ nnz, float* __restrict__ resid) {
  const long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= *total) return;
  const long long i = list[k];
  for (int m = 0; m < s; ++m) {
    idx[i * s + m] = iF[k * s + m];
    coef[i * s + m] = cF[k * s + m];
  }
  nnz[i] = nF[k];
  resid[i] = rF[k];
}

}  // namespace lrn

static int restricted_launch(const float* X, long long N, const float* D32p, const float* G, int K,
                             const uint16_t* cand, int m, int s, float eps, uint16_t* idx,
                             float* coef, uint8_t* nnz, float* resid, uint32_t* status,
                             cudaStream_t st) {
  using namespace lrn;
  if (N == 0) return DLSH_OK;
  const long long per_block = static_cast<long long>(RW) * (32 / m);
  const int grid = static_cast<int>((N + per_block - 1) / per_block);
#define LAUNCH(MM, SM)                                                                     \
  restricted_omp_kernel<MM, SM><<<grid, RW * 32, 0, st>>>(X, N, D32p, G, K, cand, s, eps, idx, \
                                                          coef, nnz, resid, status)
  switch (m) {
    case 2: LAUNCH(2, 8); break;
    case 4: LAUNCH(4, 8); break;
    case 8: LAUNCH(8, 8); break;
    case 16: if (s <= 8) LAUNCH(16, 8); else LAUNCH(16, 16); break;
    case 32: if (s <= 8) LAUNCH(32, 8); else LAUNCH(32, 16); break;
    default: return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode_restricted: m must be 2, 4, 8, 16 or 32");
  }
#undef LAUNCH
  count_launches(1);
  return check_launch("dlsh_encode_restricted: launch");
}

namespace lrn {
struct Ws {
  uint32_t* status;
  void* enc;          // encoder workspace (prepared dictionary, Gram)
  void* mlpws;        // proposal workspace (packed weights)
  uint16_t* cand;     // N x m
  uint16_t* iP;       // N x s   plain / fallback codes
  float* cP;
  uint8_t* nP;
  float* rP;
  long long* list;    // N
  float* Xfb;         // N x 45
  int* part;          // blocks
  long long* total;   // 1
  unsigned long long* nfb;
};
inline size_t carve(void* base, int K, int s, long long N, int mc, Ws& w) {
  const long long m = mc;
  Carver c(base);
  w.status = c.take<uint32_t>(64);
  w.enc = c.take<uint8_t>(encode_ws_bytes(K, s, 0));
  w.mlpws = c.take<uint8_t>(propose_ws_bytes(K));
  w.cand = c.take<uint16_t>(N * m + 1);
  w.iP = c.take<uint16_t>(N * s + 1);
  w.cP = c.take<float>(N * s + 1);
  w.nP = c.take<uint8_t>(N + 1);
  w.rP = c.take<float>(N + 1);
  w.list = c.take<long long>(N + 1);
  w.Xfb = c.take<float>(N * DLSH_D + 1);
  w.part = c.take<int>((N + CB - 1) / CB + 1);
  w.total = c.take<long long>(2);
  w.nfb = c.take<unsigned long long>(2);
  return c.size();
}
}  // namespace lrn

}  // namespace dlsh

extern "C" {

size_t dlsh_mlp_propose_workspace_size(int K, int64_t N) {
  if (K < 1 || K > DLSH_MAX_K || N < 0) return 0;
  return dlsh::propose_ws_bytes(K);
}

int dlsh_mlp_propose(const void* mlp, int K, const float* X, int64_t N, int m, uint16_t* cand,
                     void* ws, size_t ws_bytes, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  if (!mlp || K < 1 || K > DLSH_MAX_K || N < 0 || (N > 0 && (!X || !cand)))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_mlp_propose: bad arguments");
  if (m != 2 && m != 4 && m != 8 && m != 16 && m != 32)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_mlp_propose: m must be 2, 4, 8, 16 or 32");
  int rc = check_workspace(ws, ws_bytes, dlsh_mlp_propose_workspace_size(K, N), "dlsh_mlp_propose");
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* status = static_cast<uint32_t*>(ws);  // the workspace opens with its status word
  DLSH_CUDA_TRY(cudaMemsetAsync(status, 0, 4, st), "dlsh_mlp_propose: reset");
  rc = propose_enqueue(mlp, K, X, N, m, cand, ws, status, st);
  if (rc) return rc;
  return finish(st, status, flags, "dlsh_mlp_propose");
}

int dlsh_encode_restricted(const float* D, int K, int d, const float* X, int64_t N,
                           const uint16_t* cand, int m, int s, float eps, uint16_t* idx,
                           float* coef, uint8_t* nnz, float* resid_sq, void* ws, size_t ws_bytes,
                           void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  if (d != DLSH_D) return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode_restricted: d must be 45");
  if (!D || K < 1 || K > DLSH_MAX_K || s < 1 || s > 16 || N < 0)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_restricted: bad sizes");
  if (m < s || m > 32) return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode_restricted: need s <= m <= 32");
  if (N > 0 && (!X || !cand || !idx || !coef || !nnz || !resid_sq))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_restricted: NULL array");
  if (!(eps >= 0.f)) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_restricted: eps < 0");
  int rc = check_workspace(ws, ws_bytes, encode_ws_bytes(K, s, 0), "dlsh_encode_restricted");
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const float* D32p = nullptr;
  const float* G = nullptr;
  uint32_t* status = nullptr;
  rc = encode_prepare_only(D, K, s, 0, ws, st, &D32p, &G, &status);
  if (rc) return rc;
  rc = restricted_launch(X, N, D32p, G, K, cand, m, s, eps, idx, coef, nnz, resid_sq, status, st);
  if (rc) return rc;
  return finish(st, status, flags, "dlsh_encode_restricted");
}

// The candidate count: m = 0 means 2s; otherwise 2, 4, 8, 16 or 32 with s <= m.
static int learned_m(int s, int m) {
  if (m == 0) m = 2 * s;
  if (m < s || m > 32 || (m & (m - 1)) != 0 || m < 2) return 0;
  return m;
}

size_t dlsh_encode_learned_workspace_size(int K, int d, int s, int64_t N, int m) {
  if (d != DLSH_D || K < 1 || K > DLSH_MAX_K || s < 1 || s > 16 || N < 0) return 0;
  if (dlsh::encode_ws_bytes(K, s, 0) == 0 || learned_m(s, m) == 0) return 0;
  dlsh::lrn::Ws w;
  return dlsh::lrn::carve(nullptr, K, s, N, learned_m(s, m), w);
}

int dlsh_encode_learned(const float* D, int K, int d, const float* X, int64_t N, int s, float eps,
                        const void* mlp, int m_req, int mode, float tau, int fallback_precision,
                        uint16_t* idx, float* coef, uint8_t* nnz, float* resid_sq,
                        unsigned long long* n_fallback, void* ws, size_t ws_bytes, void* stream,
                        int flags) {
  using namespace dlsh;
  using namespace dlsh::lrn;
  clear_error();
  const int m = learned_m(s, m_req);
  if (m == 0)
    return set_error(DLSH_ERR_UNSUPPORTED,
                     "dlsh_encode_learned: m = %d with s = %d (need 2s <= 32 for m = 0, else m in "
                     "{2, 4, 8, 16, 32}, m >= s)", m_req, s);
  const size_t need = dlsh_encode_learned_workspace_size(K, d, s, N, m);
  if (need == 0 || !mlp || !D) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_learned: bad sizes");
  if (mode != 0 && mode != 1) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_learned: mode 0 or 1");
  if (fallback_precision < 0 || fallback_precision > 4)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_learned: unknown fallback precision");
  if (N > 0 && (!X || !idx || !coef || !nnz || !resid_sq || !n_fallback))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_learned: NULL array");
  if (!(eps >= 0.f) || !(tau >= 0.f))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_encode_learned: eps and tau must be >= 0");
  int rc = check_workspace(ws, ws_bytes, need, "dlsh_encode_learned");
  if (rc) return rc;
  Ws w;
  carve(ws, K, s, N, m, w);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DLSH_CUDA_TRY(cudaMemsetAsync(w.nfb, 0, sizeof(unsigned long long), st), "dlsh_encode_learned: reset");
  const float* D32p = nullptr;
  const float* G = nullptr;
  uint32_t* status = nullptr;
  rc = encode_prepare_only(D, K, s, 0, w.enc, st, &D32p, &G, &status);
  if (rc) return rc;
  rc = propose_enqueue(mlp, K, X, N, m, w.cand, w.mlpws, status, st);
  if (rc) return rc;
  rc = restricted_launch(X, N, D32p, G, K, w.cand, m, s, eps, idx, coef, nnz, resid_sq, status, st);
  if (rc) return rc;
  if (N > 0) {
    if (mode == 0) {
      uint32_t* est = nullptr;
      rc = encode_enqueue(D, K, X, N, s, eps, fallback_precision, w.iP, w.cP, w.nP, w.rP, w.enc, st,
                          &est);
      if (rc) return rc;
      choose_kernel<<<static_cast<int>((N + 255) / 256), 256, 0, st>>>(
          N, s, resid_sq, w.rP, w.iP, w.cP, w.nP, idx, coef, nnz, resid_sq, w.nfb);
      count_launches(1);
    } else {
      const int nb = static_cast<int>((N + CB - 1) / CB);
      const float tau2 = tau * tau;
      fb_count_kernel<<<nb, CB, 0, st>>>(resid_sq, N, tau2, w.part);
      fb_scan_kernel<<<1, 1, 0, st>>>(w.part, nb, w.total);
      fb_compact_kernel<<<nb, CB, 0, st>>>(resid_sq, X, N, tau2, w.part, w.list, w.Xfb);
      count_launches(3);
      uint32_t* est = nullptr;
      rc = encode_enqueue(D, K, w.Xfb, N, s, eps, fallback_precision, w.iP, w.cP, w.nP, w.rP,
                          w.enc, st, &est, nullptr, w.total);
      if (rc) return rc;
      fb_scatter_kernel<<<static_cast<int>((N + 255) / 256), 256, 0, st>>>(
          w.list, w.total, s, w.iP, w.cP, w.nP, w.rP, idx, coef, nnz, resid_sq);
      DLSH_CUDA_TRY(cudaMemcpyAsync(w.nfb, w.total, sizeof(long long), cudaMemcpyDeviceToDevice, st),
                    "dlsh_encode_learned: count");
      count_launches(1);
    }
  }
  DLSH_CUDA_TRY(cudaMemcpyAsync(n_fallback, w.nfb, sizeof(unsigned long long),
                                cudaMemcpyDeviceToDevice, st),
                "dlsh_encode_learned: count");
  return finish(st, status, flags, "dlsh_encode_learned");
}

// tau such that falling back whenever ||r_learned|| > tau keeps the combined
// RMSE within `max_ratio` of plain OMP's on this calibration set (host search
// over the sorted learned residuals; the smallest fallback set wins).
int dlsh_calibrate_fallback(const float* resid_learned, const float* resid_plain, int64_t N,
                            float max_ratio, float* tau, void* stream) {
  using namespace dlsh;
  clear_error();
  if (N < 1 || !resid_learned || !resid_plain || !tau || !(max_ratio >= 1.f))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_calibrate_fallback: bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<float> rl(N), rp(N);
  DLSH_CUDA_TRY(cudaMemcpyAsync(rl.data(), resid_learned, N * sizeof(float), cudaMemcpyDeviceToHost, st),
                "dlsh_calibrate_fallback: copy");
  DLSH_CUDA_TRY(cudaMemcpyAsync(rp.data(), resid_plain, N * sizeof(float), cudaMemcpyDeviceToHost, st),
                "dlsh_calibrate_fallback: copy");
  DLSH_CUDA_TRY(cudaStreamSynchronize(st), "dlsh_calibrate_fallback: sync");
  double plain = 0.0, learned = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    plain += rp[i];
    learned += std::max(rl[i], 0.f);
  }
  const double budget = plain * static_cast<double>(max_ratio) * max_ratio;
  std::vector<int64_t> order(N);
  for (int64_t i = 0; i < N; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return rl[a] > rl[b] || (rl[a] == rl[b] && a < b);
  });
  // fall back on the k largest learned residuals, k = 0, 1, ...
  double total = learned;
  int64_t k = 0;
  while (k < N && total > budget) {
    const int64_t i = order[k];
    total += static_cast<double>(rp[i]) - std::max(rl[i], 0.f);
    ++k;
  }
  // tau sits just below the last learned residual that falls back
  *tau = k >= N ? 0.f : std::sqrt(std::max(rl[order[k]], 0.f));
  return DLSH_OK;
}

}  // extern "C"
