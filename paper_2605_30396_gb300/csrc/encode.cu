// Batch-OMP sparse coding on the Blackwell tensor cores (Sec. 2.1: OMP against
// the learned dictionary, one greedy atom at a time, least squares re-fit).
//
// One CTA owns a tile of 128 signals (one per TMEM lane) and runs the s OMP
// iterations of the tile to completion; CTAs are persistent over tiles.
//   warp 5  TMA producer: streams the dictionary operand (pre-packed in the
//           canonical no-swizzle UMMA layout) into a ring of shared-memory
//           stages with cp.async.bulk; when the whole dictionary fits, it is
//           loaded once and stays resident.
//   warp 4  MMA issuer: per iteration and per chunk of BN atoms, one thread
//           issues tcgen05.mma R(128 x 48) . D_chunk^T into a TMEM buffer
//           (512 columns = 512/BN buffers, so MMAs run ahead of the epilogue).
//   warps 0-3  epilogue/solver, thread i = signal i = TMEM lane i: reads its
//           row of correlations with tcgen05.ld, keeps the running argmax
//           (exact for FP32; top-4 with an FP32 re-score for BF16/FP8),
//           extends the Cholesky factor of the support's Gram matrix, solves
//           the least-squares system, recomputes r = x - D_I gamma in FP32 and
//           writes r back as the next A operand.
// Correlation precisions: FP32 (3xTF32 split hi*hi + hi*lo + lo*hi, FP32
// accumulate), BF16, FP8 E4M3 with per-row and per-atom scales.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "host.hpp"

namespace dlsh {
namespace enc {

constexpr int TILE_M = 128;
constexpr int DPAD = 48;  // FP32 copy of D: rows padded from 45 to 48 floats
constexpr int NEPI = 128;
constexpr int NTHREADS = 192;
constexpr int SMEM_LIMIT = 232448;  // 227 KB opt-in dynamic shared memory per CTA
constexpr float CORR_STOP_REL = 1e-7f;
constexpr float PIVOT_MIN = 1e-6f;
constexpr float FP8_MAX = 448.f;

// 16-byte K-blocks per operand row and operand parts, per precision.
__host__ __device__ constexpr int op_kb(int prec) { return prec == 0 ? 12 : (prec == 1 ? 6 : 4); }
__host__ __device__ constexpr int op_parts(int prec) { return prec == 0 ? 2 : 1; }

struct Plan {
  int prec, BN, K, Kp, nchunks, stages, resident, s;
  uint32_t a_bytes, chunk_bytes;
  uint32_t off_a, off_ring, off_x, off_L, off_sel, off_y, off_g, off_sig, off_bar, smem;
};

inline int choose_bn(int prec, int s) { return (prec == 0 && s > 8) ? 64 : 128; }

int make_plan(int K, int s, int prec, Plan& p, int smem_limit = SMEM_LIMIT) {
  p.prec = prec;
  p.K = K;
  p.s = s;
  p.BN = choose_bn(prec, s);
  p.nchunks = (K + p.BN - 1) / p.BN;
  p.Kp = p.nchunks * p.BN;
  p.a_bytes = TILE_M * op_kb(prec) * 16 * op_parts(prec);
  p.chunk_bytes = p.BN * op_kb(prec) * 16 * op_parts(prec);
  uint32_t off = 0;
  auto take = [&](uint32_t bytes) {
    uint32_t o = (off + 1023u) & ~1023u;
    off = o + bytes;
    return o;
  };
  p.off_a = take(p.a_bytes);
  p.off_x = take(DPAD * TILE_M * 4);
  p.off_L = take(static_cast<uint32_t>(s * (s + 1) / 2) * TILE_M * 4);
  p.off_sel = take(s * TILE_M * 4);
  p.off_y = take(s * TILE_M * 4);
  p.off_g = take(s * TILE_M * 4);
  p.off_sig = take(prec == 2 ? p.Kp * 4 : 0);
  p.off_bar = take(1024);
  const uint32_t fixed = (off + 1023u) & ~1023u;
  if (fixed >= static_cast<uint32_t>(smem_limit)) return DLSH_ERR_UNSUPPORTED;
  int fit = static_cast<int>((smem_limit - fixed) / p.chunk_bytes);
  if (fit > 32) fit = 32;
  p.stages = fit < p.nchunks ? fit : p.nchunks;
  if (p.stages < 1 || (p.stages < 2 && p.nchunks > 1)) return DLSH_ERR_UNSUPPORTED;
  p.resident = p.stages >= p.nchunks;
  p.off_ring = fixed;
  p.smem = fixed + p.stages * p.chunk_bytes;
  // keep one CTA per SM: TMEM (512 columns) is allocated whole by each CTA
  if (p.smem < 120 * 1024) p.smem = 120 * 1024;
  return DLSH_OK;
}

struct Args {
  const float* X;
  int64_t N;
  const float* D32p;    // Kp x 48 FP32 (zero padded)
  const float* G;       // K x K FP32 Gram matrix D D^T
  const uint8_t* img;   // nchunks x chunk_bytes, packed UMMA operand images
  const float* sigma;   // Kp per-atom FP8 scales
  uint16_t* idx;
  float* coef;
  uint8_t* nnz;
  float* resid_sq;
  float eps;
  uint32_t* status;
  long long budget;
  Plan p;
};

// ---------------------------------------------------------------------------
// Operand packing.  A row (signal i) occupies 16 bytes per K-block at
// kb * (128*16) + i*16: core matrices of 8 rows x 16 bytes, LBO = 2048 bytes
// along K, SBO = 128 bytes between 8-row groups.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return lo | (hi << 16);
}

// Writes row i of the A operand from r[48] (FP32).  Returns the FP8 row scale
// (1 for the other precisions).
template <int PREC>
__device__ __forceinline__ float write_a_row(uint8_t* A, int i, const float (&r)[48]) {
  constexpr uint32_t LBO = TILE_M * 16;
  if constexpr (PREC == 1) {
#pragma unroll
    for (int kb = 0; kb < 6; ++kb) {
      uint4 pk;
      pk.x = pack_bf16x2(r[8 * kb + 0], r[8 * kb + 1]);
      pk.y = pack_bf16x2(r[8 * kb + 2], r[8 * kb + 3]);
      pk.z = pack_bf16x2(r[8 * kb + 4], r[8 * kb + 5]);
      pk.w = pack_bf16x2(r[8 * kb + 6], r[8 * kb + 7]);
      *reinterpret_cast<uint4*>(A + kb * LBO + i * 16) = pk;
    }
    return 1.f;
  } else if constexpr (PREC == 0) {
    constexpr uint32_t PART = TILE_M * 12 * 16;
#pragma unroll
    for (int kb = 0; kb < 12; ++kb) {
      float4 hi, lo;
      hi.x = to_tf32(r[4 * kb + 0]);
      hi.y = to_tf32(r[4 * kb + 1]);
      hi.z = to_tf32(r[4 * kb + 2]);
      hi.w = to_tf32(r[4 * kb + 3]);
      lo.x = to_tf32(r[4 * kb + 0] - hi.x);
      lo.y = to_tf32(r[4 * kb + 1] - hi.y);
      lo.z = to_tf32(r[4 * kb + 2] - hi.z);
      lo.w = to_tf32(r[4 * kb + 3] - hi.w);
      *reinterpret_cast<float4*>(A + kb * LBO + i * 16) = hi;
      *reinterpret_cast<float4*>(A + PART + kb * LBO + i * 16) = lo;
    }
    return 1.f;
  } else {
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < 48; ++k) mx = fmaxf(mx, fabsf(r[k]));
    const float rho = mx > 0.f ? mx / FP8_MAX : 1.f;
    const float inv = 1.f / rho;
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
      uint4 pk;
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = 16 * kb + 4 * q;  // 48 real (zero-padded) values, then 16 zeros
        w[q] = k < 48 ? pack_e4m3x4(r[k] * inv, r[k + 1] * inv, r[k + 2] * inv, r[k + 3] * inv)
                      : 0u;
      }
      pk.x = w[0];
      pk.y = w[1];
      pk.z = w[2];
      pk.w = w[3];
      *reinterpret_cast<uint4*>(A + kb * LBO + i * 16) = pk;
    }
    return rho;
  }
}

// Issues the MMAs of one chunk: D[tmem] = A . B^T over K = 48 (64 for FP8).
// Each instruction covers 32 bytes of K (two K-blocks).
template <int PREC, int BN>
__device__ __forceinline__ void issue_chunk(uint32_t tmem_d, uint32_t a_addr, uint32_t b_addr) {
  constexpr int KB = op_kb(PREC);
  constexpr uint32_t A_LBO = TILE_M * 16, B_LBO = BN * 16, SBO = 128;
  constexpr int NKS = KB / 2;
  if constexpr (PREC == 0) {
    constexpr uint32_t idesc = umma_idesc(2, 2, TILE_M, BN);
    constexpr uint32_t A_PART = TILE_M * KB * 16, B_PART = BN * KB * 16;
#pragma unroll
    for (int pass = 0; pass < 3; ++pass) {
      const uint32_t ao = pass == 2 ? A_PART : 0u;  // lo(r) . hi(D)
      const uint32_t bo = pass == 1 ? B_PART : 0u;  // hi(r) . lo(D)
#pragma unroll
      for (int ks = 0; ks < NKS; ++ks) {
        const uint64_t ad = umma_smem_desc(a_addr + ao + ks * 2 * A_LBO, A_LBO, SBO);
        const uint64_t bd = umma_smem_desc(b_addr + bo + ks * 2 * B_LBO, B_LBO, SBO);
        umma_tf32(tmem_d, ad, bd, idesc, (pass | ks) != 0);
      }
    }
  } else {
    constexpr uint32_t idesc = PREC == 1 ? umma_idesc(1, 1, TILE_M, BN) : umma_idesc(0, 0, TILE_M, BN);
#pragma unroll
    for (int ks = 0; ks < NKS; ++ks) {
      const uint64_t ad = umma_smem_desc(a_addr + ks * 2 * A_LBO, A_LBO, SBO);
      const uint64_t bd = umma_smem_desc(b_addr + ks * 2 * B_LBO, B_LBO, SBO);
      if constexpr (PREC == 1)
        umma_bf16(tmem_d, ad, bd, idesc, ks != 0);
      else
        umma_f8(tmem_d, ad, bd, idesc, ks != 0);
    }
  }
}

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
// The encoder.
// ---------------------------------------------------------------------------
template <int PREC, int BN>
__global__ void __launch_bounds__(NTHREADS, 1) encode_kernel(const __grid_constant__ Args a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int NBUF = 512 / BN;
  const Plan& p = a.p;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s = p.s, K = p.K, nchunks = p.nchunks;
  const int ntiles = static_cast<int>((a.N + TILE_M - 1) / TILE_M);

  uint64_t* bar_a = reinterpret_cast<uint64_t*>(smem + p.off_bar);
  uint64_t* bar_full = bar_a + 1;
  uint64_t* bar_empty = bar_full + NBUF;
  uint64_t* bar_dfull = bar_empty + NBUF;
  uint64_t* bar_dempty = bar_dfull + p.stages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_dempty + p.stages);

  if (tid == 0) {
    mbar_init(bar_a, NEPI);
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&bar_full[b], 1);
      mbar_init(&bar_empty[b], NEPI);
    }
    for (int q = 0; q < p.stages; ++q) {
      mbar_init(&bar_dfull[q], 1);
      mbar_init(&bar_dempty[q], 1);
    }
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
  const uint32_t a_addr = smem_u32(smem + p.off_a);
  const uint32_t ring_addr = smem_u32(smem + p.off_ring);

  if (warp == 5) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      if (p.resident) {
        for (int c = 0; c < nchunks; ++c) {
          mbar_arrive_expect_tx(&bar_dfull[c], p.chunk_bytes);
          bulk_g2s(smem + p.off_ring + static_cast<size_t>(c) * p.chunk_bytes,
                   a.img + static_cast<size_t>(c) * p.chunk_bytes, p.chunk_bytes, &bar_dfull[c]);
        }
      } else {
        long long ring = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
          for (int it = 0; it < s && ok; ++it) {
            for (int c = 0; c < nchunks; ++c, ++ring) {
              const int st = static_cast<int>(ring % p.stages);
              const uint32_t par = static_cast<uint32_t>((ring / p.stages) & 1) ^ 1u;
              if (!mbar_wait(&bar_dempty[st], par, a.budget)) {
                flag_status(a.status, ST_TIMEOUT);
                ok = false;
                break;
              }
              mbar_arrive_expect_tx(&bar_dfull[st], p.chunk_bytes);
              bulk_g2s(smem + p.off_ring + static_cast<size_t>(st) * p.chunk_bytes,
                       a.img + static_cast<size_t>(c) * p.chunk_bytes, p.chunk_bytes,
                       &bar_dfull[st]);
            }
          }
        }
        // drain: the last release of every stage has arrived
        for (long long f = ring > p.stages ? ring - p.stages : 0; ok && f < ring; ++f) {
          if (!mbar_wait(&bar_dempty[f % p.stages], static_cast<uint32_t>((f / p.stages) & 1),
                         a.budget)) {
            flag_status(a.status, ST_TIMEOUT);
            ok = false;
          }
        }
      }
    }
  } else if (warp == 4) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t a_phase = 0;
      long long cc = 0, ring = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int it = 0; it < s && ok; ++it) {
          if (!mbar_wait(bar_a, a_phase, a.budget)) {
            flag_status(a.status, ST_TIMEOUT);
            ok = false;
            break;
          }
          a_phase ^= 1u;
          tc_fence_after();
          for (int c = 0; c < nchunks; ++c, ++cc) {
            int st;
            uint32_t dpar;
            if (p.resident) {
              st = c;
              dpar = 0;
            } else {
              st = static_cast<int>(ring % p.stages);
              dpar = static_cast<uint32_t>((ring / p.stages) & 1);
            }
            const int buf = static_cast<int>(cc % NBUF);
            const uint32_t epar = static_cast<uint32_t>((cc / NBUF) & 1) ^ 1u;
            if (!mbar_wait(&bar_dfull[st], dpar, a.budget) ||
                !mbar_wait(&bar_empty[buf], epar, a.budget)) {
              flag_status(a.status, ST_TIMEOUT);
              ok = false;
              break;
            }
            tc_fence_after();
            issue_chunk<PREC, BN>(tmem_base + buf * BN, a_addr,
                                  ring_addr + static_cast<uint32_t>(st) * p.chunk_bytes);
            tc_commit(&bar_full[buf]);
            if (!p.resident) {
              tc_commit(&bar_dempty[st]);
              ++ring;
            }
          }
        }
      }
    }
  } else {
    // ------------------------------------------------ epilogue / solver
    const int i = tid;
    uint8_t* A = smem + p.off_a;
    float* xs = reinterpret_cast<float*>(smem + p.off_x);
    float* Ls = reinterpret_cast<float*>(smem + p.off_L);
    int* sel = reinterpret_cast<int*>(smem + p.off_sel);
    float* ys = reinterpret_cast<float*>(smem + p.off_y);
    float* gs = reinterpret_cast<float*>(smem + p.off_g);
    const float* sig = reinterpret_cast<const float*>(smem + p.off_sig);
    float* sig_w = reinterpret_cast<float*>(smem + p.off_sig);
    if constexpr (PREC == 2) {
      for (int j = i; j < p.Kp; j += NEPI) sig_w[j] = a.sigma[j];
    }
    // rows 45..47 of the signal tile are padding and stay zero
    for (int k = DLSH_D; k < DPAD; ++k) xs[k * TILE_M + i] = 0.f;
#define LS(r, c) Ls[(((r) * ((r) + 1)) / 2 + (c)) * TILE_M + i]
    long long cc = 0;
    bool ok = true;
    const float eps2 = a.eps * a.eps;
    const uint32_t trow = tmem_base + (static_cast<uint32_t>(warp * 32) << 16);
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int64_t g0 = static_cast<int64_t>(tile) * TILE_M;
      const int rows = static_cast<int>(a.N - g0 < TILE_M ? a.N - g0 : TILE_M);
      named_bar_sync(1, NEPI);
      const float* Xt = a.X + g0 * DLSH_D;
      for (int f = i; f < TILE_M * DLSH_D; f += NEPI) {
        const int row = f / DLSH_D, col = f - row * DLSH_D;
        xs[col * TILE_M + row] = row < rows ? __ldg(Xt + f) : 0.f;
      }
      named_bar_sync(1, NEPI);
      float r[48];
      float xn2 = 0.f;
#pragma unroll
      for (int k = 0; k < 48; ++k) {
        r[k] = k < DLSH_D ? xs[k * TILE_M + i] : 0.f;
        xn2 = fmaf(r[k], r[k], xn2);
      }
      const float xnorm = sqrtf(xn2);
      float rn2 = xn2;
      bool active = i < rows;
      int t = 0;
      write_a_row<PREC>(A, i, r);
      fence_proxy_async_smem();
      mbar_arrive(bar_a);

      for (int it = 0; it < s; ++it) {
        if (active && rn2 <= eps2) active = false;
        // -------- atom selection over all chunks
        float tv[4] = {-1.f, -1.f, -1.f, -1.f};
        int tj[4] = {-1, -1, -1, -1};
        float bval = 0.f;
        for (int c = 0; c < nchunks; ++c, ++cc) {
          const int buf = static_cast<int>(cc % NBUF);
          if (!mbar_wait(&bar_full[buf], static_cast<uint32_t>((cc / NBUF) & 1), a.budget)) {
            flag_status(a.status, ST_TIMEOUT);
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll 1
          for (int cb = 0; cb < BN; cb += 32) {
            float v[32];
            __syncwarp();
            tmem_ld32(trow + static_cast<uint32_t>(buf * BN + cb), v);
            const int j0 = c * BN + cb;
            if constexpr (PREC == 2) {
#pragma unroll
              for (int k = 0; k < 32; ++k) v[k] *= sig[j0 + k];
            }
            float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
#pragma unroll
            for (int k = 0; k < 32; k += 4) {
              m0 = fmaxf(m0, fabsf(v[k]));
              m1 = fmaxf(m1, fabsf(v[k + 1]));
              m2 = fmaxf(m2, fabsf(v[k + 2]));
              m3 = fmaxf(m3, fabsf(v[k + 3]));
            }
            const float m = fmaxf(fmaxf(m0, m1), fmaxf(m2, m3));
            const float thr = (PREC == 0) ? tv[0] : tv[3];
            if (active && m > thr) {
#pragma unroll
              for (int k = 0; k < 32; ++k) {
                const float av = fabsf(v[k]);
                const int j = j0 + k;
                const float th = (PREC == 0) ? tv[0] : tv[3];
                if (av > th && j < K) {
                  bool taken = false;
                  for (int q = 0; q < t; ++q) taken |= (sel[q * TILE_M + i] == j);
                  if (!taken) {
                    if constexpr (PREC == 0) {
                      tv[0] = av;
                      tj[0] = j;
                      bval = v[k];
                    } else {
                      if (av > tv[0]) {
                        tv[3] = tv[2]; tj[3] = tj[2];
                        tv[2] = tv[1]; tj[2] = tj[1];
                        tv[1] = tv[0]; tj[1] = tj[0];
                        tv[0] = av; tj[0] = j;
                      } else if (av > tv[1]) {
                        tv[3] = tv[2]; tj[3] = tj[2];
                        tv[2] = tv[1]; tj[2] = tj[1];
                        tv[1] = av; tj[1] = j;
                      } else if (av > tv[2]) {
                        tv[3] = tv[2]; tj[3] = tj[2];
                        tv[2] = av; tj[2] = j;
                      } else {
                        tv[3] = av; tj[3] = j;
                      }
                    }
                  }
                }
              }
            }
          }
          tc_fence_before();
          mbar_arrive(&bar_empty[buf]);
        }
        if (!ok) break;

        if (active) {
          // -------- FP32 re-score of the low-precision candidates
          int js = tj[0];
          float best = tv[0];
          if constexpr (PREC != 0) {
            best = -1.f;
            js = -1;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (tj[q] >= 0) {
                const float4* drow = reinterpret_cast<const float4*>(a.D32p + static_cast<size_t>(tj[q]) * DPAD);
                float c0 = 0.f;
#pragma unroll
                for (int u = 0; u < 12; ++u) {
                  const float4 dv = __ldg(drow + u);
                  c0 = fmaf(r[4 * u + 0], dv.x, c0);
                  c0 = fmaf(r[4 * u + 1], dv.y, c0);
                  c0 = fmaf(r[4 * u + 2], dv.z, c0);
                  c0 = fmaf(r[4 * u + 3], dv.w, c0);
                }
                const float ac = fabsf(c0);
                if (ac > best || (ac == best && tj[q] < js)) {
                  best = ac;
                  js = tj[q];
                  bval = c0;
                }
              }
            }
          }
          (void)bval;
          if (js < 0 || !(best > CORR_STOP_REL * xnorm)) {
            active = false;
          } else {
            // -------- Cholesky update: w = L^-1 g, g_m = <d_js, d_sel[m]>
            const float* Grow = a.G + static_cast<size_t>(js) * K;
            float wn2 = 0.f;
            for (int m = 0; m < t; ++m) {
              float acc = __ldg(Grow + sel[m * TILE_M + i]);
              for (int q = 0; q < m; ++q) acc = fmaf(-LS(m, q), LS(t, q), acc);
              const float w = acc / LS(m, m);
              LS(t, m) = w;
              wn2 = fmaf(w, w, wn2);
            }
            const float gjj = __ldg(Grow + js);
            const float ell2 = gjj - wn2;
            if (!(ell2 > PIVOT_MIN * gjj)) {
              active = false;  // numerically dependent atom: not added
            } else {
              const float ell = sqrtf(ell2);
              LS(t, t) = ell;
              // b_t = <d_js, x>, forward step of L y = D_I^T x
              const float4* drow = reinterpret_cast<const float4*>(a.D32p + static_cast<size_t>(js) * DPAD);
              float b = 0.f;
#pragma unroll
              for (int u = 0; u < 12; ++u) {
                const float4 dv = __ldg(drow + u);
                b = fmaf(dv.x, xs[(4 * u + 0) * TILE_M + i], b);
                b = fmaf(dv.y, xs[(4 * u + 1) * TILE_M + i], b);
                b = fmaf(dv.z, xs[(4 * u + 2) * TILE_M + i], b);
                b = fmaf(dv.w, xs[(4 * u + 3) * TILE_M + i], b);
              }
              float yt = b;
              for (int m = 0; m < t; ++m) yt = fmaf(-LS(t, m), ys[m * TILE_M + i], yt);
              ys[t * TILE_M + i] = yt / ell;
              sel[t * TILE_M + i] = js;
              ++t;
              // back substitution L^T gamma = y
              for (int m = t - 1; m >= 0; --m) {
                float acc = ys[m * TILE_M + i];
                for (int q = m + 1; q < t; ++q) acc = fmaf(-LS(q, m), gs[q * TILE_M + i], acc);
                gs[m * TILE_M + i] = acc / LS(m, m);
              }
              // residual r = x - D_I gamma, in FP32 from the FP32 atoms
#pragma unroll
              for (int k = 0; k < 48; ++k) r[k] = k < DLSH_D ? xs[k * TILE_M + i] : 0.f;
              for (int m = 0; m < t; ++m) {
                const float gm = gs[m * TILE_M + i];
                const float4* dr = reinterpret_cast<const float4*>(a.D32p + static_cast<size_t>(sel[m * TILE_M + i]) * DPAD);
#pragma unroll
                for (int u = 0; u < 12; ++u) {
                  const float4 dv = __ldg(dr + u);
                  r[4 * u + 0] = fmaf(-gm, dv.x, r[4 * u + 0]);
                  r[4 * u + 1] = fmaf(-gm, dv.y, r[4 * u + 1]);
                  r[4 * u + 2] = fmaf(-gm, dv.z, r[4 * u + 2]);
                  r[4 * u + 3] = fmaf(-gm, dv.w, r[4 * u + 3]);
                }
              }
              rn2 = 0.f;
#pragma unroll
              for (int k = 0; k < 48; ++k) rn2 = fmaf(r[k], r[k], rn2);
            }
          }
        }
        if (it + 1 < s) {
          if (active) write_a_row<PREC>(A, i, r);
          fence_proxy_async_smem();
          mbar_arrive(bar_a);
        }
      }
      if (!ok) break;
      if (i < rows) {
        const int64_t g = g0 + i;
        for (int m = 0; m < s; ++m) {
          a.idx[g * s + m] = m < t ? static_cast<uint16_t>(sel[m * TILE_M + i]) : static_cast<uint16_t>(0);
          a.coef[g * s + m] = m < t ? gs[m * TILE_M + i] : 0.f;
        }
        a.nnz[g] = static_cast<uint8_t>(t);
        if (a.resid_sq) a.resid_sq[g] = rn2;
      }
    }
#undef LS
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
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
  if (prec < 0 || prec > 2)
    return set_error(DLSH_ERR_INVALID_ARG, "%s: unknown precision %d", call, prec);
  if (!D) return set_error(DLSH_ERR_INVALID_ARG, "%s: D is NULL", call);
  return DLSH_OK;
}

template <int PREC, int BN>
static int launch_encode(const Args& a, int grid, cudaStream_t st) {
  auto fn = encode_kernel<PREC, BN>;
  DLSH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT),
                "dlsh_encode: cudaFuncSetAttribute");
  fn<<<grid, NTHREADS, a.p.smem, st>>>(a);
  count_launches(1);
  return check_launch("dlsh_encode: launch");
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

// Entry points shared with the learning loop (learn.cu).
int encode_enqueue(const float* D, int K, const float* X, int64_t N, int s, float eps, int prec,
                   uint16_t* idx, float* coef, uint8_t* nnz, float* resid_sq, void* ws,
                   cudaStream_t st, uint32_t** status_out) {
  using namespace enc;
  Plan p;
  if (make_plan(K, s, prec, p) != DLSH_OK)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_encode: K=%d s=%d precision=%d does not fit", K,
                     s, prec);
  Ws w;
  carve(ws, p, w);
  if (status_out) *status_out = w.status;
  int rc = prepare(D, p, w, true, st);
  if (rc) return rc;
  if (N == 0) return DLSH_OK;
  Args a;
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
  a.p = p;
  const int ntiles = static_cast<int>((N + TILE_M - 1) / TILE_M);
  int sms = device_sm_count();
  if (sms <= 0) sms = 1;
  const int grid = ntiles < sms ? ntiles : sms;
  if (p.BN == 128) {
    if (prec == 0) return launch_encode<0, 128>(a, grid, st);
    if (prec == 1) return launch_encode<1, 128>(a, grid, st);
    return launch_encode<2, 128>(a, grid, st);
  }
  return launch_encode<0, 64>(a, grid, st);
}

size_t encode_ws_bytes(int K, int s, int prec) {
  enc::Plan p;
  if (enc::make_plan(K, s, prec, p) != DLSH_OK) return 0;
  enc::Ws w;
  return enc::carve(nullptr, p, w);
}

}  // namespace dlsh

extern "C" {

size_t dlsh_encode_workspace_size(int K, int d, int s, int precision) {
  if (d != DLSH_D || K < 1 || K > DLSH_MAX_K || s < 1 || s > 16 || precision < 0 || precision > 2)
    return 0;
  return dlsh::encode_ws_bytes(K, s, precision);
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
  rc = encode_enqueue(D, K, X, N, s, eps, precision, idx, coef, nnz, resid_sq, ws, st, &status);
  if (rc) return rc;
  return finish(st, status, flags, "dlsh_encode");
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
    if (precision == 0) rc = launch_correlate<0, 128>(R, M, p, w, C, grid, st);
    else if (precision == 1) rc = launch_correlate<1, 128>(R, M, p, w, C, grid, st);
    else rc = launch_correlate<2, 128>(R, M, p, w, C, grid, st);
    if (rc) return rc;
  }
  return finish(st, w.status, flags, "dlsh_correlate");
}

}  // extern "C"
