// Learned support proposal: a 45 -> 256 -> 256 -> K MLP (GELU, BF16 weights,
// FP32 accumulation) trained on (signal, OMP support) pairs that the codec
// itself produces, whose 2s largest logits name candidate atoms for an OMP
// restricted to them; plain OMP (Sec. 2.1) remains the fallback.
//
// GPU design:
//   gemm_kernel     tcgen05 BF16 GEMM, C = A B^T with FP32 accumulation in TMEM.
//                   Operands are read with arbitrary row/column strides (so
//                   transposed activations need no copies) and staged into the
//                   canonical no-swizzle K-major layout (cp.async 16-byte copies
//                   where a row's 8 k values are contiguous, else by the
//                   threads); three shared-memory stages keep the loads two
//                   k-tiles ahead of the MMAs.  Epilogues: store (split-K partials), +bias,
//                   +bias with GELU (stores the pre-activation for backward).
//   small kernels   input normalisation, BCE-with-logits gradient and loss,
//                   GELU backward, bias gradients, split-K reduction, Adam.
// Inference (the logits, or the m best atoms per signal) is one fused kernel
// (propose.cu); the layer-by-layer forward here serves training.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "host.hpp"
#include "internal.hpp"
#include "mlp.cuh"

namespace dlsh {
namespace mlp {

constexpr int GM = 128;  // tile rows = MMA M
constexpr int GN = 128;  // tile cols = MMA N
constexpr int GK = 64;   // k-tile: four MMAs of K = 16
constexpr int GT = 128;  // threads per GEMM CTA
constexpr int NS = 3;    // operand stages (loads run NS - 1 k-tiles ahead)
constexpr uint32_t A_STAGE = GM * GK * 2;  // 16 KB
constexpr uint32_t B_STAGE = GN * GK * 2;  // 16 KB

enum : int { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2 };

struct Mat {
  const __nv_bfloat16* p;
  long long srow, scol;  // element (r, c) at p[r * srow + c * scol]
};

struct GemmArgs {
  Mat A;  // M x Kd
  Mat B;  // N x Kd
  int M, N, Kd;
  int klen;            // k range per split (multiple of GK)
  float* C;            // M x N (row stride ldc), split z at C + z * zstride
  long long ldc, zstride;
  const float* bias;   // N (EPI_BIAS, EPI_BIAS_GELU)
  __nv_bfloat16* H;    // GELU output, M x N (row stride ldh)
  long long ldh;
  int epi;
  uint32_t* status;
  long long budget;
};

// Stages rows [r0, r0+rows_tile) x k-range [k0, k0+GK) of X into the canonical
// layout at `dst` (16-byte K-blocks: byte (kk/8) * rows_tile*16 + r*16 + (kk%8)*2).
template <int ROWS>
__device__ __forceinline__ void stage_tile(uint8_t* dst, const Mat& X, int r0, int nrows, int k0,
                                           int kend) {
  const int t = threadIdx.x;
  const bool kvec = X.scol == 1 && (X.srow % 8) == 0 && (reinterpret_cast<uintptr_t>(X.p) % 16) == 0;
  const bool rvec = X.srow == 1 && (X.scol % 8) == 0 && (reinterpret_cast<uintptr_t>(X.p) % 16) == 0;
  if (kvec) {
    // chunk = 8 consecutive k of one row; consecutive threads take consecutive rows
    for (int c = t; c < ROWS * (GK / 8); c += GT) {
      const int kb = c / ROWS, r = c - kb * ROWS;
      const int row = r0 + r, k = k0 + kb * 8;
      uint8_t* d = dst + kb * (ROWS * 16) + r * 16;
      if (row < nrows && k + 8 <= kend) {
        // asynchronous 16-byte copy, completed by the caller's cp.async wait
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(d)),
                     "l"(X.p + static_cast<long long>(row) * X.srow + k)
                     : "memory");
      } else {
        uint4 v = make_uint4(0, 0, 0, 0);
        if (row < nrows && k < kend) {
          const __nv_bfloat16* src = X.p + static_cast<long long>(row) * X.srow + k;
          __nv_bfloat16 tmp[8];
          for (int e = 0; e < 8; ++e) tmp[e] = (k + e < kend) ? src[e] : __float2bfloat16(0.f);
          v = *reinterpret_cast<uint4*>(tmp);
        }
        *reinterpret_cast<uint4*>(d) = v;
      }
    }
  } else if (rvec) {
    // chunk = 8 consecutive rows at one k; scattered into 8 core-matrix rows
    for (int c = t; c < (ROWS / 8) * GK; c += GT) {
      const int kk = c / (ROWS / 8), rc = c - kk * (ROWS / 8);
      const int row = r0 + rc * 8, k = k0 + kk;
      __nv_bfloat16 tmp[8];
      if (k < kend && row + 8 <= nrows) {
        *reinterpret_cast<uint4*>(tmp) =
            *reinterpret_cast<const uint4*>(X.p + row + static_cast<long long>(k) * X.scol);
      } else {
        for (int e = 0; e < 8; ++e)
          tmp[e] = (k < kend && row + e < nrows) ? X.p[row + e + static_cast<long long>(k) * X.scol]
                                                 : __float2bfloat16(0.f);
      }
      uint8_t* base = dst + (kk >> 3) * (ROWS * 16) + (kk & 7) * 2;
      for (int e = 0; e < 8; ++e)
        *reinterpret_cast<__nv_bfloat16*>(base + (rc * 8 + e) * 16) = tmp[e];
    }
  } else {
    for (int c = t; c < ROWS * GK; c += GT) {
      const int kk = c / ROWS, r = c - kk * ROWS;
      const int row = r0 + r, k = k0 + kk;
      const __nv_bfloat16 v = (row < nrows && k < kend)
                                  ? X.p[static_cast<long long>(row) * X.srow + static_cast<long long>(k) * X.scol]
                                  : __float2bfloat16(0.f);
      *reinterpret_cast<__nv_bfloat16*>(dst + (kk >> 3) * (ROWS * 16) + r * 16 + (kk & 7) * 2) = v;
    }
  }
}

__global__ void __launch_bounds__(GT) gemm_kernel(const __grid_constant__ GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* As = smem;                        // NS stages
  uint8_t* Bs = smem + NS * A_STAGE;         // NS stages
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NS * (A_STAGE + B_STAGE));
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + NS);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
  const int kbeg = blockIdx.z * g.klen;
  const int kend = kbeg + g.klen < g.Kd ? kbeg + g.klen : g.Kd;
  const int nkt = kend > kbeg ? (kend - kbeg + GK - 1) / GK : 0;
  if (tid == 0) {
    for (int q = 0; q < NS; ++q) mbar_init(&bar[q], 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, GN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = umma_idesc(1, 1, GM, GN);
  auto stage = [&](int t) {
    const int sl = t % NS, k0 = kbeg + t * GK;
    stage_tile<GM>(As + sl * A_STAGE, g.A, m0, g.M, k0, kend);
    stage_tile<GN>(Bs + sl * B_STAGE, g.B, n0, g.N, k0, kend);
  };
  // k-tile t lands in slot t % NS; its MMAs' completion is phase t / NS of that
  // slot's barrier.  Loads run NS - 1 tiles ahead of the MMAs.
  for (int t = 0; t < NS - 1; ++t) {
    if (t < nkt) stage(t);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  bool ok = true;
  for (int nk = 0; nk < nkt; ++nk) {
    const int nx = nk + NS - 1;
    if (nx < nkt && nk >= 1) {  // the slot's previous tile (nk - 1) must be consumed
      const int tp = nk - 1;
      if (!mbar_wait(&bar[tp % NS], static_cast<uint32_t>((tp / NS) & 1), g.budget)) {
        flag_status(g.status, ST_TIMEOUT);
        ok = false;
      }
    }
    if (__syncthreads_or(!ok)) break;
    if (nx < nkt) stage(nx);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group %0;" ::"n"(NS - 1) : "memory");  // tile nk has landed
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const int sl = nk % NS;
      const uint32_t a = smem_u32(As + sl * A_STAGE), b = smem_u32(Bs + sl * B_STAGE);
#pragma unroll
      for (int ks = 0; ks < GK / 16; ++ks) {
        const uint64_t ad = umma_smem_desc(a + ks * 2 * (GM * 16), GM * 16, 128);
        const uint64_t bd = umma_smem_desc(b + ks * 2 * (GN * 16), GN * 16, 128);
        umma_bf16(tmem, ad, bd, idesc, (nk > 0 || ks > 0) ? 1u : 0u);
      }
      tc_commit(&bar[sl]);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // drain: the last tile's commit completes after every earlier MMA
  if (ok && nkt > 0) {
    const int tl = nkt - 1;
    if (!mbar_wait(&bar[tl % NS], static_cast<uint32_t>((tl / NS) & 1), g.budget)) {
      flag_status(g.status, ST_TIMEOUT);
      ok = false;
    }
  }
  const int nk = nkt;
  __syncthreads();
  tc_fence_after();
  // Epilogue: each warp moves its 32 rows x 32 columns from TMEM through a
  // padded shared-memory tile, so every global store writes 32 consecutive
  // columns of one row (the operand stages are free once the MMAs are done).
  float* stg = reinterpret_cast<float*>(smem) + warp * 32 * 33;
  if (ok) {
    for (int cb = 0; cb < GN; cb += 32) {
      float v[32];
      __syncwarp();
      if (nk > 0) {
        tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + cb, v);
      } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = 0.f;
      }
#pragma unroll
      for (int k = 0; k < 32; ++k) stg[lane * 33 + k] = v[k];
      __syncwarp();
      const int col = n0 + cb + lane;
      const float bcol = (g.epi != EPI_STORE && col < g.N) ? g.bias[col] : 0.f;
      for (int r = 0; r < 32; ++r) {
        const int row = m0 + warp * 32 + r;
        if (row < g.M && col < g.N) {
          const float z = add_bias(stg[r * 33 + lane], bcol);
          if (g.C)
            g.C[static_cast<long long>(blockIdx.z) * g.zstride + static_cast<long long>(row) * g.ldc + col] = z;
          if (g.epi == EPI_BIAS_GELU)
            g.H[static_cast<long long>(row) * g.ldh + col] = __float2bfloat16(gelu_f(z));
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, GN);
  }
}

}  // namespace mlp
}  // namespace dlsh

namespace dlsh {
namespace mlp {

// ---- input: xn = x / ||x|| (0 if x = 0), padded to 64 columns, BF16 ---------
__global__ void normalize_kernel(const float* __restrict__ X, long long n, __nv_bfloat16* __restrict__ Xn) {
  const long long i = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const float x0 = X[i * DLSH_D + lane];
  const float x1 = lane < DLSH_D - 32 ? X[i * DLSH_D + 32 + lane] : 0.f;
  __nv_bfloat16 y0, y1;
  normalise_pair(x0, x1, y0, y1);
  Xn[i * XIN + lane] = y0;
  Xn[i * XIN + 32 + lane] = y1;
}

// ---- BCE-with-logits gradient (mean over B*K) and per-row loss ----------------
// dZ (FP32, in place of Z) and a BF16 copy; y = 1 on the row's support atoms.
__global__ void bce_grad_kernel(float* __restrict__ Z, __nv_bfloat16* __restrict__ dZb, int K,
                                const uint16_t* __restrict__ idx, const uint8_t* __restrict__ nnz,
                                int s, float inv_bk, double* __restrict__ row_loss) {
  __shared__ double red[256];
  __shared__ int sup[32];
  __shared__ int nz_s;
  const long long b = blockIdx.x;
  if (threadIdx.x == 0) nz_s = nnz[b] > s ? s : nnz[b];
  if (static_cast<int>(threadIdx.x) < s) sup[threadIdx.x] = idx[b * s + threadIdx.x];
  __syncthreads();
  const int nz = nz_s;
  double acc = 0.0;
  float* zr = Z + b * K;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const float z = zr[k];
    bool y = false;
    for (int t = 0; t < nz; ++t) y |= (sup[t] == k);
    const float sg = 1.f / (1.f + expf(-z));
    const float g = (sg - (y ? 1.f : 0.f)) * inv_bk;
    acc += static_cast<double>(fmaxf(z, 0.f) - (y ? z : 0.f) + log1pf(expf(-fabsf(z))));
    zr[k] = g;
    dZb[b * K + k] = __float2bfloat16(g);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (static_cast<int>(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) row_loss[b] = red[0];
}

// mean loss = sum(row_loss) / (B K), fixed-order reduction
__global__ void loss_kernel(const double* __restrict__ row_loss, int B, double inv_bk, float* out) {
  __shared__ double red[1024];
  double acc = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) acc += row_loss[b];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (static_cast<int>(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = static_cast<float>(red[0] * inv_bk);
}

// dZ = dH * gelu'(Z) (FP32 in place of dH) and a BF16 copy
__global__ void gelu_bwd_kernel(float* __restrict__ dH, const float* __restrict__ Z,
                                __nv_bfloat16* __restrict__ dZb, long long n) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = dH[i] * gelu_grad_f(Z[i]);
  dH[i] = g;
  dZb[i] = __float2bfloat16(g);
}

// column sums of an R x C FP32 matrix, two levels in a fixed order
constexpr int CS_ROWS = 256;
__global__ void colsum_partial_kernel(const float* __restrict__ A, int R, int C,
                                      float* __restrict__ part) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r0 = blockIdx.y * CS_ROWS;
  if (c >= C) return;
  float acc = 0.f;
  for (int r = r0; r < r0 + CS_ROWS && r < R; ++r) acc += A[static_cast<long long>(r) * C + c];
  part[static_cast<long long>(blockIdx.y) * C + c] = acc;
}
__global__ void colsum_final_kernel(const float* __restrict__ part, int nparts, int C,
                                    float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  float acc = 0.f;
  for (int p = 0; p < nparts; ++p) acc += part[static_cast<long long>(p) * C + c];
  out[c] = acc;
}

// out[i] = sum_z part[z][i] (split-K reduction in a fixed order)
__global__ void splitk_reduce_kernel(const float* __restrict__ part, int splits, long long n,
                                     float* __restrict__ out) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc = 0.f;
  for (int z = 0; z < splits; ++z) acc += part[static_cast<long long>(z) * n + i];
  out[i] = acc;
}

// Adam on every parameter; refreshes the BF16 mirror.
__global__ void adam_kernel(float* __restrict__ P, float* __restrict__ m1, float* __restrict__ m2,
                            __nv_bfloat16* __restrict__ Pb, const float* __restrict__ G, long long n,
                            float lr, float beta1, float beta2, float eps, float bc1, float bc2) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float a = beta1 * m1[i] + (1.f - beta1) * g;
  const float v = beta2 * m2[i] + (1.f - beta2) * g * g;
  m1[i] = a;
  m2[i] = v;
  const float p = P[i] - lr * (a / bc1) / (sqrtf(v / bc2) + eps);
  P[i] = p;
  Pb[i] = __float2bfloat16(p);
}

__global__ void mirror_kernel(const float* __restrict__ P, __nv_bfloat16* __restrict__ Pb, long long n) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) Pb[i] = __float2bfloat16(P[i]);
}

}  // namespace mlp
}  // namespace dlsh

// ===========================================================================
// Host side
// ===========================================================================
namespace dlsh {
namespace mlp {

constexpr int SPLIT_K = 1024;  // batch rows per split of the weight-gradient GEMMs

static int gemm(const Mat& A, const Mat& B, int M, int N, int Kd, float* C, long long ldc, int epi,
                const float* bias, __nv_bfloat16* H, long long ldh, int splits, long long zstride,
                uint32_t* status, cudaStream_t st) {
  static PerDevice<int> attr;
  int attr_ok = 0;
  const int arc = attr.get(&attr_ok, [](int& v) {
    DLSH_CUDA_TRY(cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       NS * (A_STAGE + B_STAGE) + 64),
                  "dlsh_mlp: attribute");
    v = 1;
    return DLSH_OK;
  });
  if (arc) return arc;
  GemmArgs g;
  g.A = A;
  g.B = B;
  g.M = M;
  g.N = N;
  g.Kd = Kd;
  const int kt = (Kd + GK - 1) / GK;
  const int per = (kt + splits - 1) / splits;
  g.klen = per * GK;
  g.C = C;
  g.ldc = ldc;
  g.zstride = zstride;
  g.bias = bias;
  g.H = H;
  g.ldh = ldh;
  g.epi = epi;
  g.status = status;
  g.budget = kWaitBudget;
  dim3 grid((N + GN - 1) / GN, (M + GM - 1) / GM, splits);
  gemm_kernel<<<grid, GT, NS * (A_STAGE + B_STAGE) + 64, st>>>(g);
  count_launches(1);
  return check_launch("dlsh_mlp: gemm");
}

// Training / forward workspace for batches of up to B rows.
struct TWs {
  uint32_t* status;
  __nv_bfloat16* Xn;   // B x 64
  float* Z1;           // B x 256 (then dZ1)
  float* Z2;           // B x 256 (then dZ2)
  __nv_bfloat16* H1;   // B x 256
  __nv_bfloat16* H2;   // B x 256
  float* Z3;           // B x K (logits, then dZ3)
  __nv_bfloat16* dZ3b; // B x K
  float* dH;           // B x 256 (dH2 / dH1)
  __nv_bfloat16* dZb;  // B x 256
  float* part;         // split-K partials / column-sum partials
  float* grads;        // parameter gradients
  double* row_loss;    // B
  float* loss;         // 1
};

static size_t carve_t(void* base, int K, long long B, TWs& w) {
  const Layout L = layout(K);
  const long long splits = (B + SPLIT_K - 1) / SPLIT_K;
  const long long part = std::max<long long>(splits * std::max<long long>(static_cast<long long>(K) * HID, HID * HID),
                                             ((B + CS_ROWS - 1) / CS_ROWS) * std::max(K, HID));
  Carver c(base);
  w.status = c.take<uint32_t>(64);
  w.Xn = c.take<__nv_bfloat16>(B * XIN);
  w.Z1 = c.take<float>(B * HID);
  w.Z2 = c.take<float>(B * HID);
  w.H1 = c.take<__nv_bfloat16>(B * HID);
  w.H2 = c.take<__nv_bfloat16>(B * HID);
  w.Z3 = c.take<float>(B * K);
  w.dZ3b = c.take<__nv_bfloat16>(B * K);
  w.dH = c.take<float>(B * HID);
  w.dZb = c.take<__nv_bfloat16>(B * HID);
  w.part = c.take<float>(part);
  w.grads = c.take<float>(L.n);
  w.row_loss = c.take<double>(B);
  w.loss = c.take<float>(4);
  return c.size();
}

static inline Mat rowmajor(const __nv_bfloat16* p, long long ld) { return Mat{p, ld, 1}; }
static inline Mat transposed(const __nv_bfloat16* p, long long ld) { return Mat{p, 1, ld}; }

// Training forward through the three layers: logits in w.Z3 (B x K), hidden
// pre-activations in w.Z1 / w.Z2 for the backward pass.
static int forward(const Blob& b, int K, const float* X, long long B, const TWs& w, cudaStream_t st) {
  const Layout L = layout(K);
  normalize_kernel<<<static_cast<int>((B + 7) / 8), 256, 0, st>>>(X, B, w.Xn);
  count_launches(1);
  int rc = gemm(rowmajor(w.Xn, XIN), rowmajor(b.Pb + L.W1, XIN), B, HID, XIN,
                w.Z1, HID, EPI_BIAS_GELU, b.P + L.b1, w.H1, HID, 1, 0,
                w.status, st);
  if (rc) return rc;
  rc = gemm(rowmajor(w.H1, HID), rowmajor(b.Pb + L.W2, HID), B, HID, HID, w.Z2,
            HID, EPI_BIAS_GELU, b.P + L.b2, w.H2, HID, 1, 0, w.status, st);
  if (rc) return rc;
  return gemm(rowmajor(w.H2, HID), rowmajor(b.Pb + L.W3, HID), B, K, HID, w.Z3, K, EPI_BIAS,
              b.P + L.b3, nullptr, 0, 1, 0, w.status, st);
}

static int colsum(const float* A, int R, int C, float* out, float* part, cudaStream_t st) {
  const int parts = (R + CS_ROWS - 1) / CS_ROWS;
  colsum_partial_kernel<<<dim3((C + 255) / 256, parts), 256, 0, st>>>(A, R, C, part);
  colsum_final_kernel<<<(C + 255) / 256, 256, 0, st>>>(part, parts, C, out);
  count_launches(2);
  return check_launch("dlsh_mlp: colsum");
}

// dW = dZ^T A_in over the batch (split-K, reduced in a fixed order)
static int weight_grad(const __nv_bfloat16* dZb, int Nout, const __nv_bfloat16* Ain, int Nin,
                       long long B, float* out, float* part, uint32_t* status, cudaStream_t st) {
  const int splits = static_cast<int>((B + SPLIT_K - 1) / SPLIT_K);
  const long long n = static_cast<long long>(Nout) * Nin;
  int rc = gemm(transposed(dZb, Nout), transposed(Ain, Nin), Nout, Nin, static_cast<int>(B), part,
                Nin, EPI_STORE, nullptr, nullptr, 0, splits, n, status, st);
  if (rc) return rc;
  splitk_reduce_kernel<<<static_cast<int>((n + 255) / 256), 256, 0, st>>>(part, splits, n, out);
  count_launches(1);
  return check_launch("dlsh_mlp: split-K reduce");
}

// forward + backward: parameter gradients in w.grads, mean loss in w.loss
static int gradients(const Blob& b, int K, const float* X, long long B, const uint16_t* idx,
                     const uint8_t* nnz, int s, const TWs& w, cudaStream_t st) {
  const Layout L = layout(K);
  int rc = forward(b, K, X, B, w, st);
  if (rc) return rc;
  const float inv_bk = static_cast<float>(1.0 / (static_cast<double>(B) * K));
  bce_grad_kernel<<<static_cast<int>(B), 256, 0, st>>>(w.Z3, w.dZ3b, K, idx, nnz, s, inv_bk,
                                                       w.row_loss);
  loss_kernel<<<1, 1024, 0, st>>>(w.row_loss, static_cast<int>(B), 1.0 / (static_cast<double>(B) * K),
                                  w.loss);
  count_launches(2);
  // layer 3
  rc = weight_grad(w.dZ3b, K, w.H2, HID, B, w.grads + L.W3, w.part, w.status, st);
  if (rc) return rc;
  rc = colsum(w.Z3, static_cast<int>(B), K, w.grads + L.b3, w.part, st);
  if (rc) return rc;
  rc = gemm(rowmajor(w.dZ3b, K), transposed(b.Pb + L.W3, HID), B, HID, K, w.dH, HID, EPI_STORE,
            nullptr, nullptr, 0, 1, 0, w.status, st);
  if (rc) return rc;
  const long long nh = B * HID;
  gelu_bwd_kernel<<<static_cast<int>((nh + 255) / 256), 256, 0, st>>>(w.dH, w.Z2, w.dZb, nh);
  count_launches(1);
  // layer 2 (dZ2 now in w.dH / w.dZb)
  rc = weight_grad(w.dZb, HID, w.H1, HID, B, w.grads + L.W2, w.part, w.status, st);
  if (rc) return rc;
  rc = colsum(w.dH, static_cast<int>(B), HID, w.grads + L.b2, w.part, st);
  if (rc) return rc;
  rc = gemm(rowmajor(w.dZb, HID), transposed(b.Pb + L.W2, HID), B, HID, HID, w.Z2, HID, EPI_STORE,
            nullptr, nullptr, 0, 1, 0, w.status, st);  // dH1 into the Z2 buffer (no longer needed)
  if (rc) return rc;
  gelu_bwd_kernel<<<static_cast<int>((nh + 255) / 256), 256, 0, st>>>(w.Z2, w.Z1, w.dZb, nh);
  count_launches(1);
  // layer 1 (dZ1 now in w.Z2 / w.dZb)
  rc = weight_grad(w.dZb, HID, w.Xn, XIN, B, w.grads + L.W1, w.part, w.status, st);
  if (rc) return rc;
  return colsum(w.Z2, static_cast<int>(B), HID, w.grads + L.b1, w.part, st);
}

static int adam(const Blob& b, int K, const float* grads, float lr, long long step,
                cudaStream_t st) {
  const Layout L = layout(K);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float bc1 = static_cast<float>(1.0 - pow(0.9, static_cast<double>(step)));
  const float bc2 = static_cast<float>(1.0 - pow(0.999, static_cast<double>(step)));
  adam_kernel<<<static_cast<int>((L.n + 255) / 256), 256, 0, st>>>(b.P, b.m1, b.m2, b.Pb, grads, L.n, lr,
                                                                    b1, b2, eps, bc1, bc2);
  count_launches(1);
  return check_launch("dlsh_mlp: adam");
}

}  // namespace mlp

size_t mlp_train_ws_bytes(int K, long long B) {
  mlp::TWs w;
  return mlp::carve_t(nullptr, K, B, w);
}

}  // namespace dlsh

extern "C" {

long long dlsh_mlp_num_params(int K) { return K >= 1 ? dlsh::mlp::layout(K).n : 0; }

size_t dlsh_mlp_size(int K) {
  if (K < 1 || K > DLSH_MAX_K) return 0;
  dlsh::mlp::Blob b;
  return dlsh::mlp::carve_blob(nullptr, K, b);
}

size_t dlsh_mlp_workspace_size(int K, int64_t B) {
  if (K < 1 || K > DLSH_MAX_K || B < 1) return 0;
  return std::max(dlsh::mlp_train_ws_bytes(K, B), dlsh::propose_ws_bytes(K));
}

int dlsh_mlp_init(void* mlp, int K, const float* params, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  if (!mlp || !params || K < 1 || K > DLSH_MAX_K)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_mlp_init: bad arguments");
  if (reinterpret_cast<uintptr_t>(mlp) % 256)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_mlp_init: blob must be 256-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mlp::Blob b;
  mlp::carve_blob(mlp, K, b);
  const long long n = mlp::layout(K).n;
  DLSH_CUDA_TRY(cudaMemcpyAsync(b.P, params, n * sizeof(float), cudaMemcpyDeviceToDevice, st),
                "dlsh_mlp_init: copy");
  DLSH_CUDA_TRY(cudaMemsetAsync(b.m1, 0, n * sizeof(float), st), "dlsh_mlp_init: m1");
  DLSH_CUDA_TRY(cudaMemsetAsync(b.m2, 0, n * sizeof(float), st), "dlsh_mlp_init: m2");
  DLSH_CUDA_TRY(cudaMemsetAsync(b.step, 0, 2 * sizeof(long long), st), "dlsh_mlp_init: step");
  mlp::mirror_kernel<<<static_cast<int>((n + 255) / 256), 256, 0, st>>>(b.P, b.Pb, n);
  count_launches(1);
  return finish(st, nullptr, flags, "dlsh_mlp_init");
}

int dlsh_mlp_params(const void* mlp, int K, float* params, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  if (!mlp || !params || K < 1) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_mlp_params: bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mlp::Blob b;
  mlp::carve_blob(const_cast<void*>(mlp), K, b);
  DLSH_CUDA_TRY(cudaMemcpyAsync(params, b.P, mlp::layout(K).n * sizeof(float),
                                cudaMemcpyDeviceToDevice, st),
                "dlsh_mlp_params: copy");
  return finish(st, nullptr, flags, "dlsh_mlp_params");
}

static int mlp_common_checks(const char* call, const void* mlp, int K, const float* X, int64_t B,
                             void* ws, size_t ws_bytes) {
  using namespace dlsh;
  if (!mlp || K < 1 || K > DLSH_MAX_K) return set_error(DLSH_ERR_INVALID_ARG, "%s: bad blob or K", call);
  if (B < 1 || !X) return set_error(DLSH_ERR_INVALID_ARG, "%s: bad batch", call);
  return check_workspace(ws, ws_bytes, dlsh_mlp_workspace_size(K, B), call);
}

int dlsh_mlp_forward(const void* mlp, int K, const float* X, int64_t B, float* logits, void* ws,
                     size_t ws_bytes, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  int rc = mlp_common_checks("dlsh_mlp_forward", mlp, K, X, B, ws, ws_bytes);
  if (rc) return rc;
  if (!logits) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_mlp_forward: NULL logits");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* status = static_cast<uint32_t*>(ws);  // both workspace layouts open with it
  DLSH_CUDA_TRY(cudaMemsetAsync(status, 0, 4, st), "dlsh_mlp_forward: reset");
  rc = infer_logits_enqueue(mlp, K, X, B, logits, ws, status, st);
  if (rc) return rc;
  return finish(st, status, flags, "dlsh_mlp_forward");
}

int dlsh_mlp_gradients(const void* mlp, int K, const float* X, int64_t B, const uint16_t* idx,
                       const uint8_t* nnz, int s, float* grads, float* loss, void* ws,
                       size_t ws_bytes, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  int rc = mlp_common_checks("dlsh_mlp_gradients", mlp, K, X, B, ws, ws_bytes);
  if (rc) return rc;
  if (!idx || !nnz || !grads || s < 1 || s > DLSH_MAX_S)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_mlp_gradients: bad targets");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mlp::Blob b;
  mlp::carve_blob(const_cast<void*>(mlp), K, b);
  mlp::TWs w;
  mlp::carve_t(ws, K, B, w);
  DLSH_CUDA_TRY(cudaMemsetAsync(w.status, 0, 4, st), "dlsh_mlp_gradients: reset");
  rc = mlp::gradients(b, K, X, B, idx, nnz, s, w, st);
  if (rc) return rc;
  DLSH_CUDA_TRY(cudaMemcpyAsync(grads, w.grads, sizeof(float) * mlp::layout(K).n,
                                cudaMemcpyDeviceToDevice, st),
                "dlsh_mlp_gradients: copy");
  if (loss)
    DLSH_CUDA_TRY(cudaMemcpyAsync(loss, w.loss, sizeof(float), cudaMemcpyDeviceToDevice, st),
                  "dlsh_mlp_gradients: loss");
  return finish(st, w.status, flags, "dlsh_mlp_gradients");
}

int dlsh_mlp_train_step(void* mlp, int K, const float* X, int64_t B, const uint16_t* idx,
                        const uint8_t* nnz, int s, float lr, int64_t step, float* loss, void* ws,
                        size_t ws_bytes, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  int rc = mlp_common_checks("dlsh_mlp_train_step", mlp, K, X, B, ws, ws_bytes);
  if (rc) return rc;
  if (!idx || !nnz || s < 1 || s > DLSH_MAX_S || step < 1)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_mlp_train_step: bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mlp::Blob b;
  mlp::carve_blob(mlp, K, b);
  mlp::TWs w;
  mlp::carve_t(ws, K, B, w);
  DLSH_CUDA_TRY(cudaMemsetAsync(w.status, 0, 4, st), "dlsh_mlp_train_step: reset");
  rc = mlp::gradients(b, K, X, B, idx, nnz, s, w, st);
  if (rc) return rc;
  rc = mlp::adam(b, K, w.grads, lr, step, st);
  if (rc) return rc;
  if (loss)
    DLSH_CUDA_TRY(cudaMemcpyAsync(loss, w.loss, sizeof(float), cudaMemcpyDeviceToDevice, st),
                  "dlsh_mlp_train_step: loss");
  return finish(st, w.status, flags, "dlsh_mlp_train_step");
}

int dlsh_mlp_train(void* mlp, int K, const float* X, int64_t N, const uint16_t* idx,
                   const uint8_t* nnz, int s, int epochs, int64_t batch, float lr,
                   float* loss_per_step, void* ws, size_t ws_bytes, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  if (batch < 1 || N < batch || epochs < 1)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_mlp_train: need epochs >= 1 and N >= batch >= 1");
  int rc = mlp_common_checks("dlsh_mlp_train", mlp, K, X, batch, ws, ws_bytes);
  if (rc) return rc;
  if (!idx || !nnz || s < 1 || s > DLSH_MAX_S)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_mlp_train: bad targets");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mlp::Blob b;
  mlp::carve_blob(mlp, K, b);
  mlp::TWs w;
  mlp::carve_t(ws, K, batch, w);
  DLSH_CUDA_TRY(cudaMemsetAsync(w.status, 0, 4, st), "dlsh_mlp_train: reset");
  const long long per_epoch = N / batch;
  const long long total = per_epoch * epochs;
  long long step = 0;
  for (int e = 0; e < epochs; ++e) {
    for (long long q = 0; q < per_epoch; ++q) {
      ++step;
      // cosine decay from lr to 0 over all steps
      const double frac = static_cast<double>(step - 1) / static_cast<double>(total);
      const float lr_t = static_cast<float>(0.5 * lr * (1.0 + cos(M_PI * frac)));
      const long long off = q * batch;
      rc = mlp::gradients(b, K, X + off * DLSH_D, batch, idx + off * s, nnz + off, s, w, st);
      if (rc) return rc;
      rc = mlp::adam(b, K, w.grads, lr_t, step, st);
      if (rc) return rc;
      if (loss_per_step)
        DLSH_CUDA_TRY(cudaMemcpyAsync(loss_per_step + (step - 1), w.loss, sizeof(float),
                                      cudaMemcpyDeviceToDevice, st),
                      "dlsh_mlp_train: loss");
    }
  }
  return finish(st, w.status, flags, "dlsh_mlp_train");
}

}  // extern "C"
