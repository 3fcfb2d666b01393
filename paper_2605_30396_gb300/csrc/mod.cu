// Dictionary update with the codes fixed (Sec. 2.1: alternating minimisation of
// Eq. 1), read as MOD: the least-squares minimiser of sum ||x_i - D alpha_i||^2
// in D, with a small ridge so that unused atoms keep it well posed:
//   G = A A^T, B = X A^T, lambda = 1e-6 trace(G)/K,
//   D~^T = (G + lambda I)^-1 (B + lambda D_old)^T, d_j = d~_j / ||d~_j||,
//   unused atoms refilled with the worst-fit signals.
//
// GPU design (deterministic, no floating-point atomics):
//   1. count_kernel   per-tile atom histograms (integer counts)
//   2. scan_kernel    exclusive scan, atom-major, tile-minor
//   3. scatter_kernel one warp per signal tile writes (signal, coef) into the
//                     atom-major list in signal order (a counting sort)
//   4. accum_kernel   one CTA per atom: row j of G and column j of B in FP64,
//                     each warp over a fixed slice, slices summed in order
//   5. FP64 blocked Cholesky of G + lambda I (diagonal factor, panel solve,
//      trailing update), forward and backward substitution for the d RHS
//   6. normalise, then refill unused atoms (argmax passes over resid_sq)
// GB300's FP64 rate is low but K^3/3 at K <= 2048 is a few GFLOP; the solve
// stays in FP64 because G + lambda I can have condition numbers near 1e6+.
#include <math.h>

#include "common.cuh"
#include "host.hpp"

namespace dlsh {
namespace mod {

constexpr int TS = 2048;       // signals per counting-sort tile
constexpr int NB = 32;         // Cholesky block
constexpr int RW = 48;         // padded RHS width (45 used)
constexpr int MAX_K = 4096;    // shared-memory G-row partials and FP64 G size limit
constexpr double RIDGE_REL = 1e-6;

struct Ws {
  uint32_t* status;
  int* cnt;        // K x T
  int* off;        // K x T
  int* atom_start; // K + 1
  int* list_sig;   // N*s
  float* list_coef;
  double* M;       // K x K (G, then G + lambda I, then its Cholesky factor)
  double* Z;       // K x RW (B^T + lambda D_old, then the solution)
  double* lam;     // [0] lambda
  int* dead;       // K
};

static size_t carve(void* base, int K, int s, int64_t N, Ws& w) {
  Carver c(base);
  const int64_t T = (N + TS - 1) / TS > 0 ? (N + TS - 1) / TS : 1;
  w.status = c.take<uint32_t>(64);
  w.cnt = c.take<int>(static_cast<size_t>(K) * T);
  w.off = c.take<int>(static_cast<size_t>(K) * T);
  w.atom_start = c.take<int>(K + 1);
  w.list_sig = c.take<int>(static_cast<size_t>(N) * s + 1);
  w.list_coef = c.take<float>(static_cast<size_t>(N) * s + 1);
  w.M = c.take<double>(static_cast<size_t>(K) * K);
  w.Z = c.take<double>(static_cast<size_t>(K) * RW);
  w.lam = c.take<double>(4);
  w.dead = c.take<int>(K);
  return c.size();
}

// ---- 1. per-tile histograms ------------------------------------------------
__global__ void count_kernel(const uint16_t* __restrict__ idx, const uint8_t* __restrict__ nnz,
                             int s, int64_t N, int K, int T, int* __restrict__ cnt,
                             uint32_t* status) {
  extern __shared__ int hist[];
  for (int j = threadIdx.x; j < K; j += blockDim.x) hist[j] = 0;
  __syncthreads();
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * TS;
  const int64_t i1 = i0 + TS < N ? i0 + TS : N;
  bool bad = false;
  for (int64_t e = i0 * s + threadIdx.x; e < i1 * s; e += blockDim.x) {
    const int64_t i = e / s;
    const int t = static_cast<int>(e - i * s);
    int nz = nnz[i];
    if (nz > s) {
      bad = true;
      nz = s;
    }
    if (t < nz) {
      const int j = idx[e];
      if (j < K)
        atomicAdd(&hist[j], 1);
      else
        bad = true;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < K; j += blockDim.x) cnt[static_cast<size_t>(j) * T + blockIdx.x] = hist[j];
  if (bad) flag_status(status, ST_BAD_INPUT);
}

// ---- 2. exclusive scan of cnt (atom-major) -----------------------------------
__global__ void scan_kernel(const int* __restrict__ cnt, int64_t total, int K, int T,
                            int* __restrict__ off, int* __restrict__ atom_start) {
  __shared__ long long part[1024];
  const int tid = threadIdx.x;
  const int64_t per = (total + blockDim.x - 1) / blockDim.x;
  const int64_t a = tid * per, b = a + per < total ? a + per : total;
  long long sum = 0;
  for (int64_t e = a; e < b; ++e) sum += cnt[e];
  part[tid] = sum;
  __syncthreads();
  if (tid == 0) {
    long long run = 0;
    for (int q = 0; q < static_cast<int>(blockDim.x); ++q) {
      const long long v = part[q];
      part[q] = run;
      run += v;
    }
  }
  __syncthreads();
  long long run = part[tid];
  for (int64_t e = a; e < b; ++e) {
    off[e] = static_cast<int>(run);
    if (e % T == 0) atom_start[e / T] = static_cast<int>(run);
    run += cnt[e];
  }
  if (tid == static_cast<int>(blockDim.x) - 1) atom_start[K] = static_cast<int>(run);
}

// ---- 3. counting-sort scatter, one warp per tile, signal order ---------------
__global__ void scatter_kernel(const uint16_t* __restrict__ idx, const float* __restrict__ coef,
                               const uint8_t* __restrict__ nnz, int s, int64_t N, int K, int T,
                               const int* __restrict__ off, int* __restrict__ list_sig,
                               float* __restrict__ list_coef) {
  extern __shared__ int cursor[];
  const int lane = threadIdx.x;
  const int b = blockIdx.x;
  for (int j = lane; j < K; j += 32) cursor[j] = off[static_cast<size_t>(j) * T + b];
  __syncwarp();
  const int64_t i0 = static_cast<int64_t>(b) * TS;
  const int64_t i1 = i0 + TS < N ? i0 + TS : N;
  for (int64_t i = i0; i < i1; ++i) {
    int nz = nnz[i];
    nz = nz > s ? s : nz;
    if (lane < nz) {
      const int j = idx[i * s + lane];
      if (j < K) {
        const int pos = atomicAdd(&cursor[j], 1);  // distinct atoms per signal: no contention
        list_sig[pos] = static_cast<int>(i);
        list_coef[pos] = coef[i * s + lane];
      }
    }
    __syncwarp();
  }
}

// ---- 4. G row j and B column j in FP64 ----------------------------------------
// 4 warps; warp w takes the w-th contiguous quarter of atom j's list; within a
// warp entries are processed in list order.  Partials are summed in warp order.
constexpr int ACC_WARPS = 4;
constexpr int BATCH = 32;

__global__ void __launch_bounds__(ACC_WARPS * 32)
    accum_kernel(const float* __restrict__ X, const uint16_t* __restrict__ idx,
                 const float* __restrict__ coef, const uint8_t* __restrict__ nnz, int s, int K,
                 const int* __restrict__ atom_start, const int* __restrict__ list_sig,
                 const float* __restrict__ list_coef, double* __restrict__ M,
                 double* __restrict__ Z) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int j = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* grow = reinterpret_cast<double*>(smraw) + static_cast<size_t>(warp) * K;
  double* bpart = reinterpret_cast<double*>(smraw) + static_cast<size_t>(ACC_WARPS) * K +
                  warp * RW;
  float* xst = reinterpret_cast<float*>(reinterpret_cast<double*>(smraw) +
                                        static_cast<size_t>(ACC_WARPS) * K + ACC_WARPS * RW) +
               warp * (BATCH * DLSH_D + BATCH * 32 * 2 + BATCH * 2);
  uint32_t* cst_i = reinterpret_cast<uint32_t*>(xst + BATCH * DLSH_D);
  float* cst_c = reinterpret_cast<float*>(cst_i + BATCH * 32);
  int* est_i = reinterpret_cast<int*>(cst_c + BATCH * 32);
  float* est_a = reinterpret_cast<float*>(est_i + BATCH);
  for (int k = lane; k < K; k += 32) grow[k] = 0.0;
  double b0 = 0.0, b1 = 0.0;
  const int e0 = atom_start[j], e1 = atom_start[j + 1];
  const int len = e1 - e0;
  const int q0 = e0 + static_cast<int>(static_cast<long long>(len) * warp / ACC_WARPS);
  const int q1 = e0 + static_cast<int>(static_cast<long long>(len) * (warp + 1) / ACC_WARPS);
  __syncwarp();
  for (int qb = q0; qb < q1; qb += BATCH) {
    const int nb = q1 - qb < BATCH ? q1 - qb : BATCH;
    if (lane < nb) {
      est_i[lane] = list_sig[qb + lane];
      est_a[lane] = list_coef[qb + lane];
    }
    __syncwarp();
    // stage the batch's signals and codes
    for (int f = lane; f < nb * DLSH_D; f += 32) {
      const int e = f / DLSH_D, dd = f - e * DLSH_D;
      xst[f] = X[static_cast<int64_t>(est_i[e]) * DLSH_D + dd];
    }
    for (int f = lane; f < nb * s; f += 32) {
      const int e = f / s, t = f - e * s;
      const int64_t i = est_i[e];
      const int nz = nnz[i];
      cst_i[e * 32 + t] = t < nz ? idx[i * s + t] : 0xFFFFFFFFu;
      cst_c[e * 32 + t] = coef[i * s + t];
    }
    __syncwarp();
    for (int e = 0; e < nb; ++e) {
      const double a = est_a[e];
      if (lane < s) {
        const uint32_t k = cst_i[e * 32 + lane];
        if (k < static_cast<uint32_t>(K)) grow[k] += a * static_cast<double>(cst_c[e * 32 + lane]);
      }
      b0 += a * static_cast<double>(xst[e * DLSH_D + lane]);
      if (lane < DLSH_D - 32) b1 += a * static_cast<double>(xst[e * DLSH_D + 32 + lane]);
      __syncwarp();
    }
  }
  bpart[lane] = b0;
  if (lane < RW - 32) bpart[32 + lane] = lane < DLSH_D - 32 ? b1 : 0.0;
  __syncthreads();
  double* gw = reinterpret_cast<double*>(smraw);
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double acc = 0.0;
    for (int w = 0; w < ACC_WARPS; ++w) acc += gw[static_cast<size_t>(w) * K + k];
    M[static_cast<size_t>(j) * K + k] = acc;
  }
  double* bw = reinterpret_cast<double*>(smraw) + static_cast<size_t>(ACC_WARPS) * K;
  for (int q = threadIdx.x; q < RW; q += blockDim.x) {
    double acc = 0.0;
    for (int w = 0; w < ACC_WARPS; ++w) acc += bw[w * RW + q];
    Z[static_cast<size_t>(j) * RW + q] = acc;
  }
}

static size_t accum_smem(int K) {
  return static_cast<size_t>(ACC_WARPS) * K * 8 + ACC_WARPS * RW * 8 +
         static_cast<size_t>(ACC_WARPS) * (BATCH * DLSH_D + BATCH * 32 * 2 + BATCH * 2) * 4;
}

// ---- 5a. lambda = 1e-6 trace(G)/K; M += lambda I; Z += lambda D_old -----------
__global__ void ridge_kernel(double* __restrict__ M, double* __restrict__ Z,
                             const float* __restrict__ D_old, int K, double* lam_out) {
  __shared__ double part[1024];
  __shared__ double lam_s;
  double acc = 0.0;
  for (int j = threadIdx.x; j < K; j += blockDim.x) acc += M[static_cast<size_t>(j) * K + j];
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int q = 0; q < static_cast<int>(blockDim.x); ++q) tr += part[q];
    lam_s = tr > 0.0 ? RIDGE_REL * tr / K : RIDGE_REL;
    *lam_out = lam_s;
  }
  __syncthreads();
  const double lam = lam_s;
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    M[static_cast<size_t>(j) * K + j] += lam;
    for (int q = 0; q < DLSH_D; ++q)
      Z[static_cast<size_t>(j) * RW + q] += lam * static_cast<double>(D_old[static_cast<size_t>(j) * DLSH_D + q]);
  }
}

// ---- 5b. blocked Cholesky (lower, in place, row-major M[r*K + c]) -------------
__global__ void potrf_diag_kernel(double* __restrict__ M, int K, int k0, uint32_t* status) {
  __shared__ double A[NB][NB + 1];
  const int nb = K - k0 < NB ? K - k0 : NB;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 32
  if (tx < nb && ty < nb) A[ty][tx] = M[static_cast<size_t>(k0 + ty) * K + k0 + tx];
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    if (tx == 0 && ty == 0) {
      double dv = A[c][c];
      if (!(dv > 0.0)) {
        flag_status(status, ST_BAD_INPUT);
        dv = 1e-300;
      }
      A[c][c] = sqrt(dv);
    }
    __syncthreads();
    if (tx == 0 && ty > c && ty < nb) A[ty][c] /= A[c][c];
    __syncthreads();
    if (ty > c && ty < nb && tx > c && tx <= ty) A[ty][tx] -= A[ty][c] * A[tx][c];
    __syncthreads();
  }
  if (tx < nb && ty < nb) M[static_cast<size_t>(k0 + ty) * K + k0 + tx] = tx <= ty ? A[ty][tx] : 0.0;
}

// Rows below the diagonal block: L21 = A21 L11^-T, one thread per row.
__global__ void trsm_panel_kernel(double* __restrict__ M, int K, int k0) {
  __shared__ double L[NB][NB + 1];
  const int nb = K - k0 < NB ? K - k0 : NB;
  for (int f = threadIdx.x; f < NB * NB; f += blockDim.x) {
    const int r = f / NB, c = f % NB;
    L[r][c] = (r < nb && c < nb) ? M[static_cast<size_t>(k0 + r) * K + k0 + c] : 0.0;
  }
  __syncthreads();
  const int row = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= K) return;
  double* mr = M + static_cast<size_t>(row) * K + k0;
  double v[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) v[c] = c < nb ? mr[c] : 0.0;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    if (c < nb) {
      double acc = v[c];
#pragma unroll
      for (int q = 0; q < c; ++q) acc -= v[q] * L[c][q];
      v[c] = acc / L[c][c];
    }
  }
#pragma unroll
  for (int c = 0; c < NB; ++c)
    if (c < nb) mr[c] = v[c];
}

// Trailing update A22 -= L21 L21^T on lower 32x32 tiles.
__global__ void syrk_kernel(double* __restrict__ M, int K, int k0) {
  const int k1 = k0 + NB;
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  __shared__ double Li[32][NB + 1];
  __shared__ double Lj[32][NB + 1];
  const int r0 = k1 + bi * 32, c0 = k1 + bj * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    Li[r][tx] = (r0 + r < K) ? M[static_cast<size_t>(r0 + r) * K + k0 + tx] : 0.0;
    Lj[r][tx] = (c0 + r < K) ? M[static_cast<size_t>(c0 + r) * K + k0 + tx] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int gr = r0 + r, gc = c0 + tx;
    if (gr < K && gc < K && gc <= gr) {
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < NB; ++q) acc += Li[r][q] * Lj[tx][q];
      M[static_cast<size_t>(gr) * K + gc] -= acc;
    }
  }
}

// ---- 5c. forward solve L y = Z, block kb (left-looking), one CTA per column ---
__global__ void fwd_block_kernel(const double* __restrict__ M, double* __restrict__ Z, int K,
                                 int k0) {
  __shared__ double y[NB];
  const int col = blockIdx.x, q = threadIdx.x;  // 32 threads
  const int nb = K - k0 < NB ? K - k0 : NB;
  if (q < nb) {
    double acc = Z[static_cast<size_t>(k0 + q) * RW + col];
    const double* lr = M + static_cast<size_t>(k0 + q) * K;
    for (int r = 0; r < k0; ++r) acc -= lr[r] * Z[static_cast<size_t>(r) * RW + col];
    y[q] = acc;
  }
  __syncthreads();
  if (q == 0) {
    for (int c = 0; c < nb; ++c) {
      double acc = y[c];
      const double* lr = M + static_cast<size_t>(k0 + c) * K + k0;
      for (int p = 0; p < c; ++p) acc -= lr[p] * y[p];
      y[c] = acc / lr[c];
    }
  }
  __syncthreads();
  if (q < nb) Z[static_cast<size_t>(k0 + q) * RW + col] = y[q];
}

// ---- 5d. backward solve L^T x = y, block kb (from the last), per column -------
__global__ void bwd_block_kernel(const double* __restrict__ M, double* __restrict__ Z, int K,
                                 int k0) {
  __shared__ double x[NB];
  const int col = blockIdx.x, q = threadIdx.x;
  const int nb = K - k0 < NB ? K - k0 : NB;
  if (q < nb) {
    double acc = Z[static_cast<size_t>(k0 + q) * RW + col];
    for (int r = k0 + nb; r < K; ++r)
      acc -= M[static_cast<size_t>(r) * K + k0 + q] * Z[static_cast<size_t>(r) * RW + col];
    x[q] = acc;
  }
  __syncthreads();
  if (q == 0) {
    for (int c = nb - 1; c >= 0; --c) {
      double acc = x[c];
      for (int p = c + 1; p < nb; ++p) acc -= M[static_cast<size_t>(k0 + p) * K + k0 + c] * x[p];
      x[c] = acc / M[static_cast<size_t>(k0 + c) * K + k0 + c];
    }
  }
  __syncthreads();
  if (q < nb) Z[static_cast<size_t>(k0 + q) * RW + col] = x[q];
}

// ---- 6a. normalise; mark dead atoms ----------------------------------------------
__global__ void normalise_kernel(const double* __restrict__ Z, const int* __restrict__ atom_start,
                                 int K, float* __restrict__ D_new, const float* __restrict__ D_old,
                                 int* __restrict__ dead) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= K) return;
  const double z0 = Z[static_cast<size_t>(j) * RW + lane];
  const double z1 = lane < DLSH_D - 32 ? Z[static_cast<size_t>(j) * RW + 32 + lane] : 0.0;
  double n2 = z0 * z0 + z1 * z1;
  for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  const bool unused = atom_start[j + 1] == atom_start[j];
  const bool isdead = unused || !(n2 > 0.0);
  if (lane == 0) dead[j] = isdead ? 1 : 0;
  const double inv = isdead ? 0.0 : 1.0 / sqrt(n2);
  float* dr = D_new + static_cast<size_t>(j) * DLSH_D;
  const float* dold = D_old + static_cast<size_t>(j) * DLSH_D;
  dr[lane] = isdead ? dold[lane] : static_cast<float>(z0 * inv);
  if (lane < DLSH_D - 32) dr[32 + lane] = isdead ? dold[32 + lane] : static_cast<float>(z1 * inv);
}

// ---- 6b. refill dead atoms in increasing j with the largest-residual signals -----
// Picks come in the order (resid desc, index asc); each pass takes the best key
// strictly after the previous pick.  Signals with x = 0 are skipped.
__global__ void __launch_bounds__(1024)
    refill_kernel(const float* __restrict__ X, const float* __restrict__ resid, int64_t N, int K,
                  const int* __restrict__ dead, float* __restrict__ D_new) {
  __shared__ float bv[1024];
  __shared__ long long bi[1024];
  __shared__ float prev_v;
  __shared__ long long prev_i;
  __shared__ int found;
  const int tid = threadIdx.x;
  if (tid == 0) {
    prev_v = INFINITY;
    prev_i = -1;
  }
  __syncthreads();
  for (int j = 0; j < K; ++j) {
    if (!dead[j]) continue;  // uniform across the block
    while (true) {
      const float pv = prev_v;
      const long long pi = prev_i;
      float best = -1.f;
      long long besti = -1;
      for (int64_t i = tid; i < N; i += blockDim.x) {
        const float v = resid[i];
        const bool after = (v < pv) || (v == pv && i > pi);
        if (after && (v > best || (v == best && (besti < 0 || i < besti)))) {
          best = v;
          besti = i;
        }
      }
      bv[tid] = best;
      bi[tid] = besti;
      __syncthreads();
      for (int w = 512; w > 0; w >>= 1) {
        if (tid < w) {
          const float v2 = bv[tid + w];
          const long long i2 = bi[tid + w];
          if (i2 >= 0 && (bi[tid] < 0 || v2 > bv[tid] || (v2 == bv[tid] && i2 < bi[tid]))) {
            bv[tid] = v2;
            bi[tid] = i2;
          }
        }
        __syncthreads();
      }
      const long long pick = bi[0];
      if (pick < 0) {
        if (tid == 0) found = 0;
        __syncthreads();
        break;
      }
      // norm of the picked signal
      if (tid < 32) {
        const float x0 = X[pick * DLSH_D + tid];
        const float x1 = tid < DLSH_D - 32 ? X[pick * DLSH_D + 32 + tid] : 0.f;
        double n2 = static_cast<double>(x0) * x0 + static_cast<double>(x1) * x1;
        for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
        if (n2 > 0.0) {
          const double inv = 1.0 / sqrt(n2);
          D_new[static_cast<size_t>(j) * DLSH_D + tid] = static_cast<float>(x0 * inv);
          if (tid < DLSH_D - 32) D_new[static_cast<size_t>(j) * DLSH_D + 32 + tid] = static_cast<float>(x1 * inv);
        }
        if (tid == 0) {
          found = n2 > 0.0 ? 1 : 2;
          prev_v = bv[0];
          prev_i = pick;
        }
      }
      __syncthreads();
      if (found == 1) break;
    }
    __syncthreads();
    if (found == 0) break;  // no signals left
  }
}

}  // namespace mod

size_t mod_ws_bytes(int K, int s, int64_t N) {
  mod::Ws w;
  return mod::carve(nullptr, K, s, N, w);
}

// Enqueues one MOD update (no host synchronisation; capturable).
int mod_enqueue(const float* X, int64_t N, int K, const uint16_t* idx, const float* coef,
                const uint8_t* nnz, int s, const float* D_old, const float* resid,
                float* D_new, void* ws, cudaStream_t st, uint32_t** status_out) {
  using namespace mod;
  Ws w;
  carve(ws, K, s, N, w);
  if (status_out) *status_out = w.status;
  DLSH_CUDA_TRY(cudaMemsetAsync(w.status, 0, sizeof(uint32_t), st), "dlsh_mod_update: reset");
  const int T = static_cast<int>((N + TS - 1) / TS > 0 ? (N + TS - 1) / TS : 1);
  if (N > 0) {
    count_kernel<<<T, 256, K * sizeof(int), st>>>(idx, nnz, s, N, K, T, w.cnt, w.status);
  } else {
    DLSH_CUDA_TRY(cudaMemsetAsync(w.cnt, 0, sizeof(int) * K * T, st), "dlsh_mod_update: cnt");
  }
  scan_kernel<<<1, 1024, 0, st>>>(w.cnt, static_cast<int64_t>(K) * T, K, T, w.off, w.atom_start);
  if (N > 0)
    scatter_kernel<<<T, 32, K * sizeof(int), st>>>(idx, coef, nnz, s, N, K, T, w.off, w.list_sig,
                                                  w.list_coef);
  const size_t asm_bytes = accum_smem(K);
  DLSH_CUDA_TRY(cudaFuncSetAttribute(accum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(asm_bytes)),
                "dlsh_mod_update: attribute");
  accum_kernel<<<K, ACC_WARPS * 32, asm_bytes, st>>>(X, idx, coef, nnz, s, K, w.atom_start,
                                                     w.list_sig, w.list_coef, w.M, w.Z);
  ridge_kernel<<<1, 1024, 0, st>>>(w.M, w.Z, D_old, K, w.lam);
  for (int k0 = 0; k0 < K; k0 += NB) {
    potrf_diag_kernel<<<1, dim3(32, 32), 0, st>>>(w.M, K, k0, w.status);
    const int rest = K - k0 - NB;
    if (rest > 0) {
      trsm_panel_kernel<<<(rest + 127) / 128, 128, 0, st>>>(w.M, K, k0);
      const int tiles = (rest + 31) / 32;
      syrk_kernel<<<dim3(tiles, tiles), dim3(32, 8), 0, st>>>(w.M, K, k0);
    }
  }
  for (int k0 = 0; k0 < K; k0 += NB) fwd_block_kernel<<<DLSH_D, 32, 0, st>>>(w.M, w.Z, K, k0);
  for (int k0 = ((K - 1) / NB) * NB; k0 >= 0; k0 -= NB)
    bwd_block_kernel<<<DLSH_D, 32, 0, st>>>(w.M, w.Z, K, k0);
  normalise_kernel<<<(K + 7) / 8, 256, 0, st>>>(w.Z, w.atom_start, K, D_new, D_old, w.dead);
  if (resid && N > 0) refill_kernel<<<1, 1024, 0, st>>>(X, resid, N, K, w.dead, D_new);
  const int nblk = (K + NB - 1) / NB;
  count_launches((N > 0 ? 3 : 1) + 3 + (3 * nblk - 2) + 2 * nblk + 1 + ((resid && N > 0) ? 1 : 0));
  return check_launch("dlsh_mod_update: launch");
}

}  // namespace dlsh

extern "C" {

size_t dlsh_mod_workspace_size(int K, int d, int s, int64_t N) {
  if (d != DLSH_D || K < 1 || K > dlsh::mod::MAX_K || s < 1 || s > DLSH_MAX_S || N < 0) return 0;
  return dlsh::mod_ws_bytes(K, s, N);
}

int dlsh_mod_update(const float* X, int64_t N, int d, int K, const uint16_t* idx,
                    const float* coef, const uint8_t* nnz, int s, const float* D_old,
                    const float* resid_sq, float* D_new, void* ws, size_t ws_bytes, void* stream,
                    int flags) {
  using namespace dlsh;
  clear_error();
  if (d != DLSH_D) return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_mod_update: d must be 45");
  if (K < 1 || K > mod::MAX_K)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_mod_update: K must be in [1, 4096], got %d", K);
  if (s < 1 || s > DLSH_MAX_S)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_mod_update: s must be in [1, 32]");
  if (N < 0 || N * s >= (1LL << 31))
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_mod_update: N*s must be < 2^31");
  if (!D_old || !D_new) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_mod_update: NULL D");
  if (N > 0 && (!X || !idx || !coef || !nnz))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_mod_update: NULL array");
  int rc = check_workspace(ws, ws_bytes, mod_ws_bytes(K, s, N), "dlsh_mod_update");
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* status = nullptr;
  rc = mod_enqueue(X, N, K, idx, coef, nnz, s, D_old, resid_sq, D_new, ws, st, &status);
  if (rc) return rc;
  return finish(st, status, flags, "dlsh_mod_update");
}

}  // extern "C"
