// Batch-OMP sparse coding on the Blackwell tensor cores (Sec. 2.1: OMP against
// the learned dictionary, one greedy atom at a time, least squares re-fit).
//
// One CTA owns a tile of 128 signals (one per TMEM lane) and runs the s OMP
// iterations of the tile to completion; CTAs are persistent over tiles.
//   warp 17  TMA producer: streams the dictionary operand (pre-packed in the
//            canonical no-swizzle UMMA layout) into a ring of shared-memory
//            stages with cp.async.bulk; when the whole dictionary fits, it is
//            loaded once and stays resident.
//   warp 16  MMA issuer: per iteration and per chunk of BN atoms, one thread
//            issues tcgen05.mma R(128 x 48) . D_chunk^T into a TMEM buffer
//            (512 columns = 512/BN buffers, so MMAs run ahead of selection).
//   warps 0-15  selection + solver, in two phases per iteration:
//            selection: four threads per TMEM lane (one per column quarter)
//            read the row's correlations with tcgen05.ld and keep the running
//            argmax on 32-bit keys (|c| and the column index);
//            solver: four sub-lanes per signal, each owning 12 of the 48 dims,
//            merge the quarters (for BF16/FP8 the four quarter winners are
//            re-scored in FP32),
//            extend the Cholesky factor of the support's Gram matrix, solve
//            the least-squares system, recompute r = x - D_I gamma in FP32 and
//            write r back as the next A operand.
// Correlation precisions: FP32 (3xTF32 split hi*hi + hi*lo + lo*hi, FP32
// accumulate), BF16, FP8 E4M3 with per-row and per-atom scales.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>

#include "common.cuh"
#include "host.hpp"
#include "internal.hpp"

namespace dlsh {
namespace enc {

constexpr int TILE_M = 128;
constexpr int DPAD = 48;  // FP32 copy of D: rows padded from 45 to 48 floats
constexpr int NEPI = 512;      // selection/solver threads (16 warps)
constexpr int NTHREADS = 576;  // + MMA warp + TMA producer warp
constexpr int SMEM_LIMIT = 232448;  // 227 KB opt-in dynamic shared memory per CTA
constexpr float CORR_STOP_REL = 1e-7f;
constexpr float PIVOT_MIN = 1e-6f;

// The solvers run one OMP step for a row whose support holds t atoms.  Active
// rows of a tile all hold t == it atoms, so a warp's active threads agree on t
// and the step can be compiled once per t as straight-line code: with_t calls
// f(IntC<t>{}) for 0 <= t < NT.
template <int V>
struct IntC {
  static constexpr int value = V;
};
template <int NT, class F>
__device__ __forceinline__ void with_t(int t, F&& f) {
  if constexpr (NT > 0) {
    if (t == NT - 1) {
      f(IntC<NT - 1>{});
      return;
    }
    with_t<NT - 1>(t, f);
  }
}
constexpr float FP8_MAX = 448.f;
// Operand-image code of the FP16-split FP32 format (prep_kernel): hi and lo
// FP16 parts of 256 * D, 6 K blocks of 8 elements each
constexpr int OPF16X2 = 3;

// 16-byte K-blocks per operand row and operand parts, per precision.
__host__ __device__ constexpr int op_kb(int prec) { return prec == 0 ? 12 : (prec == 1 || prec == 3 ? 6 : 4); }
__host__ __device__ constexpr int op_parts(int prec) { return prec == 0 || prec == 3 ? 2 : 1; }
// K-block stride of the one-tile kernel's A operand: FP16 parts get 64 bytes of
// skew, so that a half-warp's 8-byte stores (four rows, four sub-lanes of 12
// contiguous dims) fall on sixteen different bank pairs
__host__ __device__ constexpr uint32_t a_lbo(int prec) { return prec == 3 ? TILE_M * 16 + 64 : TILE_M * 16; }

struct Plan {
  int prec, top4, ib, BN, K, Kp, nchunks, stages, resident, s;
  uint32_t a_bytes, chunk_bytes;
  uint32_t off_a, off_ring, off_x, off_L, off_sel, off_y, off_g, off_idg, off_cand, off_r,
      off_sig, off_bar, smem;
};

inline int choose_bn(int prec, int s) { return (prec == 0 && s > 8) ? 64 : 128; }

// Precision codes of the C ABI: 0 FP32 (3xTF32), 1 BF16 and 2 FP8 with the
// exact low-precision top 4 re-scored in FP32, 3 BF16 and 4 FP8 with the four
// column-quarter winners re-scored in FP32.  Returns the operand precision
// (0 FP32, 1 BF16, 2 FP8) and whether the top-4 candidates are used.
inline int operand_precision(int code, int* top4) {
  if (top4) *top4 = (code == 1 || code == 2) ? 1 : 0;
  return code == 0 ? 0 : ((code == 1 || code == 3) ? 1 : 2);
}

// The choice recorded by dlsh_autotune_encode for (K, s, precision): kernel
// variant (tuned_bn; 64 / 128 for the one-tile chunk widths) and, in
// tuned_choice, 256 x the ring-stage cap (0 if none was recorded).
int tuned_bn(int K, int s, int prec);
int tuned_choice(int K, int s, int prec);

// bn = 0: the tuned width if one was recorded, else the default.  BF16 and FP8
// use 128 (the selection's key network packs 32 columns per thread).  f16: FP32
// as three FP16 products of power-of-two scaled hi / lo parts (operand format
// OPF16X2, 128-atom chunks) instead of three TF32 products.
int make_plan(int K, int s, int code, Plan& p, int bn = 0, int smem_limit = SMEM_LIMIT, bool f16 = false) {
  int prec = operand_precision(code, &p.top4);
  if (f16 && prec == 0) {
    prec = OPF16X2;
    bn = 128;
  }
  p.prec = prec;
  p.K = K;
  p.s = s;
  if (bn == 0) bn = tuned_bn(K, s, code);
  p.BN = prec != 0 ? 128 : (bn == 64 || bn == 128 ? bn : choose_bn(prec, s));
  p.nchunks = (K + p.BN - 1) / p.BN;
  p.Kp = p.nchunks * p.BN;
  // top-4 keys carry the column within the thread's quarter (chunk, then
  // column in the chunk) in their low ib bits
  p.ib = 5;
  while ((1 << (p.ib - 5)) < p.nchunks) ++p.ib;
  p.a_bytes = a_lbo(prec) * op_kb(prec) * op_parts(prec);
  p.chunk_bytes = p.BN * op_kb(prec) * 16 * op_parts(prec);
  uint32_t off = 0;
  auto take = [&](uint32_t bytes) {
    uint32_t o = (off + 1023u) & ~1023u;
    off = o + bytes;
    return o;
  };
  p.off_a = take(p.a_bytes);
  p.off_x = take(0);  // (the signal tile is read straight into registers)
  p.off_L = take(static_cast<uint32_t>(s * (s + 1) / 2) * TILE_M * 4);
  p.off_sel = take(s * TILE_M * 4);
  p.off_y = take(s * TILE_M * 4);
  p.off_g = take(s * TILE_M * 4);
  p.off_idg = take(s * TILE_M * 4);
  p.off_cand = take(p.top4 ? TILE_M * 4 * 4 * 4 : TILE_M * 4 * 8);
  p.off_r = take(prec == 0 || prec == OPF16X2 ? 0 : NEPI * 12 * 4);
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
  unsigned long long* prof;  // optional: per-phase SM cycles of thread 0 (6 counters)
  const long long* n_dev;    // optional: signal count read on the device (overrides N)
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
  } else if constexpr (PREC == OPF16X2) {
    // three FP16 products: hi.hi, hi.lo(D), lo(r).hi
    constexpr uint32_t idesc = umma_idesc(0, 0, TILE_M, BN);
    constexpr uint32_t AL = a_lbo(OPF16X2), A_PART = KB * AL, B_PART = BN * KB * 16;
#pragma unroll
    for (int pass = 0; pass < 3; ++pass) {
      const uint32_t ao = pass == 2 ? A_PART : 0u;
      const uint32_t bo = pass == 1 ? B_PART : 0u;
#pragma unroll
      for (int ks = 0; ks < NKS; ++ks) {
        const uint64_t ad = umma_smem_desc(a_addr + ao + ks * 2 * AL, AL, SBO);
        const uint64_t bd = umma_smem_desc(b_addr + bo + ks * 2 * B_LBO, B_LBO, SBO);
        umma_bf16(tmem_d, ad, bd, idesc, (pass | ks) != 0);
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
// The encoder.  Per OMP iteration of a tile:
//   phase 1 (selection): thread (warp w < 16, lane l) reads TMEM lane
//     32*(w%4) + l, i.e. row R1 of the tile, over column quarter q = w/4 of
//     every chunk, and keeps its best candidate(s) for that row and quarter;
//   phase 2 (solver): thread (warp w, lane l) serves row R2 = 8w + l/4 with
//     sub-lane u = l%4 owning signal dims [12u, 12u+12); the four sub-lanes
//     of a row run the same scalar recurrences (bitwise identical values) and
//     combine dot products with two butterfly shuffles.
// ---------------------------------------------------------------------------
// FP16 parts: the power of two 2^e that puts a row's largest |value| mx in
// [2^14, 2^15) (e = 15 for mx = 0, clamped to [-100, 100]), read from mx's
// exponent field; rinv receives 2^-(e + 8), the inverse of the correlations'
// scale (the dictionary image holds 256 D).
__device__ __forceinline__ float pow2_scale(float mx, float& rinv) {
  const int E = static_cast<int>((__float_as_uint(mx) >> 23) & 0xffu);
  int e = mx > 0.f ? 141 - E : 15;  // frexp exponent of mx is E - 126
  e = e < -100 ? -100 : (e > 100 ? 100 : e);
  rinv = __uint_as_float(static_cast<uint32_t>(119 - e) << 23);
  return __uint_as_float(static_cast<uint32_t>(127 + e) << 23);
}

// FP16 hi and lo parts (round to nearest) of four scaled values, packed two per
// word: hi = fp16(a), lo = fp16(a - hi)
__device__ __forceinline__ void split_f16x4(float a0, float a1, float a2, float a3, uint2& ph, uint2& pl) {
  const __half2 h01 = __floats2half2_rn(a0, a1), h23 = __floats2half2_rn(a2, a3);
  const float2 f01 = __half22float2(h01), f23 = __half22float2(h23);
  const __half2 l01 = __floats2half2_rn(a0 - f01.x, a1 - f01.y);
  const __half2 l23 = __floats2half2_rn(a2 - f23.x, a3 - f23.y);
  ph = make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
  pl = make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
}

template <int PREC>
__device__ __forceinline__ void write_a_part(uint8_t* A, int row, int u, const float (&r)[12],
                                             float inv_rho) {
  constexpr uint32_t LBO = TILE_M * 16;
  if constexpr (PREC == 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int e = 12 * u + 4 * k;
      uint2 pk;
      pk.x = pack_bf16x2(r[4 * k + 0], r[4 * k + 1]);
      pk.y = pack_bf16x2(r[4 * k + 2], r[4 * k + 3]);
      *reinterpret_cast<uint2*>(A + (e >> 3) * LBO + row * 16 + (e & 7) * 2) = pk;
    }
  } else if constexpr (PREC == OPF16X2) {
    // dims 12u + 4k .. 12u + 4k + 3: half ((3u + k) & 1) of K block (12u + 4k) / 8,
    // FP16 hi / lo of the scaled values (inv_rho holds the row's scale here)
    constexpr uint32_t L = a_lbo(OPF16X2), PART = 6 * L;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int e = 12 * u + 4 * k;
      const uint32_t off = static_cast<uint32_t>(e >> 3) * L + row * 16 + ((e >> 2) & 1) * 8;
      uint2 ph, pl;
      split_f16x4(r[4 * k] * inv_rho, r[4 * k + 1] * inv_rho, r[4 * k + 2] * inv_rho, r[4 * k + 3] * inv_rho,
                  ph, pl);
      *reinterpret_cast<uint2*>(A + off) = ph;
      *reinterpret_cast<uint2*>(A + PART + off) = pl;
    }
  } else if constexpr (PREC == 0) {
    constexpr uint32_t PART = TILE_M * 12 * 16;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int kb = 3 * u + k;
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
    for (int k = 0; k < 3; ++k) {
      const int e = 12 * u + 4 * k;
      const uint32_t w = pack_e4m3x4(r[4 * k] * inv_rho, r[4 * k + 1] * inv_rho,
                                     r[4 * k + 2] * inv_rho, r[4 * k + 3] * inv_rho);
      *reinterpret_cast<uint32_t*>(A + (e >> 4) * LBO + row * 16 + (e & 15)) = w;
    }
  }
}

// Butterfly over the four sub-lanes of one row (lanes 4k..4k+3).  Only those
// four lanes take part, so rows of one warp may sit on different branches.
__device__ __forceinline__ unsigned quad_mask() {
  return 0xFu << ((threadIdx.x & 31) & ~3u);
}
__device__ __forceinline__ float quad_sum(float v) {
  const unsigned m = quad_mask();
  v += __shfl_xor_sync(m, v, 1);
  v += __shfl_xor_sync(m, v, 2);
  return v;
}
__device__ __forceinline__ float quad_max(float v) {
  const unsigned m = quad_mask();
  v = fmaxf(v, __shfl_xor_sync(m, v, 1));
  v = fmaxf(v, __shfl_xor_sync(m, v, 2));
  return v;
}

template <int NC>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float (&v)[NC]);
template <>
__device__ __forceinline__ void tmem_ld_cols<32>(uint32_t taddr, float (&v)[32]) {
  tmem_ld32(taddr, v);
}
template <>
__device__ __forceinline__ void tmem_ld_cols<16>(uint32_t taddr, float (&v)[16]) {
  tmem_ld16(taddr, v);
}

template <int NC>
__device__ __forceinline__ void tmem_ld_issue(uint32_t taddr, uint32_t (&r)[NC]);
template <>
__device__ __forceinline__ void tmem_ld_issue<32>(uint32_t taddr, uint32_t (&r)[32]) {
  tmem_ld32_issue(taddr, r);
}
template <>
__device__ __forceinline__ void tmem_ld_issue<16>(uint32_t taddr, uint32_t (&r)[16]) {
  tmem_ld16_issue(taddr, r);
}
template <int NC>
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[NC]);
template <>
__device__ __forceinline__ void tmem_ld_wait<32>(uint32_t (&r)[32]) {
  tmem_ld32_wait(r);
}
template <>
__device__ __forceinline__ void tmem_ld_wait<16>(uint32_t (&r)[16]) {
  tmem_ld16_wait(r);
}

// ---------------------------------------------------------------------------
// Exact top 4 on 32-bit keys with min/max only (no branches): lists are kept
// sorted in decreasing order, a[0] >= a[1] >= a[2] >= a[3].
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void cex(T& hi, T& lo) {
  const T h = hi > lo ? hi : lo;
  const T l = hi > lo ? lo : hi;
  hi = h;
  lo = l;
}
// a := the sorted top 4 of a and b (both sorted).  The pairwise maxima of a
// and b reversed hold the top 4 as a bitonic sequence, which two
// compare-exchange stages sort.
template <class T>
__device__ __forceinline__ void merge_top4(T (&a)[4], const T (&b)[4]) {
  T m0 = a[0] > b[3] ? a[0] : b[3];
  T m1 = a[1] > b[2] ? a[1] : b[2];
  T m2 = a[2] > b[1] ? a[2] : b[1];
  T m3 = a[3] > b[0] ? a[3] : b[0];
  cex(m0, m2);
  cex(m1, m3);
  cex(m0, m1);
  cex(m2, m3);
  a[0] = m0;
  a[1] = m1;
  a[2] = m2;
  a[3] = m3;
}
// o := the sorted top 4 of k[0..7]: sorted pairs, merged into two sorted
// quads, then the top 4 of the two quads.
__device__ __forceinline__ void top4_of8(const uint32_t* k, uint32_t (&o)[4]) {
  uint32_t p[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) p[i] = k[i];
#pragma unroll
  for (int i = 0; i < 8; i += 2) cex(p[i], p[i + 1]);
  uint32_t q[2][4];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint32_t a0 = p[4 * h], a1 = p[4 * h + 1], b0 = p[4 * h + 2], b1 = p[4 * h + 3];
    const uint32_t x = min(a0, b0), y = max(a1, b1);
    q[h][0] = max(a0, b0);
    q[h][1] = max(x, y);
    q[h][2] = min(x, y);
    q[h][3] = min(a1, b1);
  }
  merge_top4(q[0], q[1]);
#pragma unroll
  for (int i = 0; i < 4; ++i) o[i] = q[0][i];
}

// SMAX: compile-time bound on s (8 or 16) for the solver's register arrays.
// T4: BF16/FP8 candidates are each row's exact low-precision top 4 (else the
// four column-quarter winners).
// FP16 parts: the scale 2^e that puts the row's largest |value| (over the four
// sub-lanes) in [2^14, 2^15), so the hi / lo parts keep FP32's 22 significant
// bits; rinv receives 2^-(e + 8), the inverse of the correlations' scale (the
// dictionary image holds 256 D).
__device__ __forceinline__ float f16_scale(const float (&v)[12], float& rinv) {
  float mx = 0.f;
#pragma unroll
  for (int q = 0; q < 12; ++q) mx = fmaxf(mx, fabsf(v[q]));
  return pow2_scale(quad_max(mx), rinv);
}

template <int PREC, int BN, int SMAX, bool T4>
__global__ void __launch_bounds__(NTHREADS, 1) encode_kernel(const __grid_constant__ Args a) {
  // FP32 (TF32 or FP16 parts): the argmax is the selection; BF16 / FP8: the
  // candidates are re-scored in FP32 against a copy of the residual
  constexpr bool EXACT = PREC == 0 || PREC == OPF16X2;
  constexpr bool RESCORE = !EXACT;
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int NBUF = 512 / BN;
  constexpr int QC = BN / 4;  // columns of one chunk read by one phase-1 thread
  constexpr int NCAND = 1;  // one candidate per thread (column quarter) and row
  static_assert(QC <= 32, "selection keys pack a 5-bit column index");
  const Plan& p = a.p;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long NS = a.n_dev ? *a.n_dev : a.N;
  const int ntiles = static_cast<int>((NS + TILE_M - 1) / TILE_M);

  uint64_t* bar_a = reinterpret_cast<uint64_t*>(smem + p.off_bar);
  uint64_t* bar_full = bar_a + 1;
  uint64_t* bar_empty = bar_full + NBUF;
  uint64_t* bar_dfull = bar_empty + NBUF;
  uint64_t* bar_dempty = bar_dfull + p.stages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_dempty + p.stages);

  if (tid == 0) {
    if (a.prof)
      for (int k = 0; k < 12; ++k)
        reinterpret_cast<unsigned long long*>(smem + p.off_bar + 928)[k] = 0;
    mbar_init(bar_a, 1);
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&bar_full[b], 1);
      mbar_init(&bar_empty[b], NEPI / 32);
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
  // optional phase profile (SM cycles), one shared-memory slot per counter:
  // 0-5 first selection/solver thread, 6-8 MMA issuer, 9 TMA producer
  unsigned long long* pcs = reinterpret_cast<unsigned long long*>(smem + p.off_bar + 928);
  const bool prof_any = a.prof != nullptr;

  if (warp == NEPI / 32 + 1) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      if (p.resident) {
        for (int c = 0; c < p.nchunks; ++c) {
          mbar_arrive_expect_tx(&bar_dfull[c], p.chunk_bytes);
          bulk_g2s(smem + p.off_ring + static_cast<size_t>(c) * p.chunk_bytes,
                   a.img + static_cast<size_t>(c) * p.chunk_bytes, p.chunk_bytes, &bar_dfull[c]);
        }
      } else {
        long long ring = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
          for (int it = 0; it < p.s && ok; ++it) {
            for (int c = 0; c < p.nchunks; ++c, ++ring) {
              const int st = static_cast<int>(ring % p.stages);
              const uint32_t par = static_cast<uint32_t>((ring / p.stages) & 1) ^ 1u;
              const long long Wp = prof_any ? clock64() : 0;
              if (!mbar_wait(&bar_dempty[st], par, a.budget)) {
                flag_status(a.status, ST_TIMEOUT);
                ok = false;
                break;
              }
              if (prof_any) pcs[9] += clock64() - Wp;
              mbar_arrive_expect_tx(&bar_dfull[st], p.chunk_bytes);
              bulk_g2s(smem + p.off_ring + static_cast<size_t>(st) * p.chunk_bytes,
                       a.img + static_cast<size_t>(c) * p.chunk_bytes, p.chunk_bytes,
                       &bar_dfull[st]);
            }
          }
        }
        for (long long f = ring > p.stages ? ring - p.stages : 0; ok && f < ring; ++f) {
          if (!mbar_wait(&bar_dempty[f % p.stages], static_cast<uint32_t>((f / p.stages) & 1),
                         a.budget)) {
            flag_status(a.status, ST_TIMEOUT);
            ok = false;
          }
        }
      }
    }
  } else if (warp == NEPI / 32) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t a_phase = 0;
      long long cc = 0, ring = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int nchunks = p.nchunks;
        for (int it = 0; it < p.s && ok; ++it) {
          const long long Wa = prof_any ? clock64() : 0;
          if (!mbar_wait(bar_a, a_phase, a.budget)) {
            flag_status(a.status, ST_TIMEOUT);
            ok = false;
            break;
          }
          if (prof_any) pcs[6] += clock64() - Wa;
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
            const long long Wd = prof_any ? clock64() : 0;
            const bool okd = mbar_wait(&bar_dfull[st], dpar, a.budget);
            const long long We = prof_any ? clock64() : 0;
            const bool oke = okd && mbar_wait(&bar_empty[buf], epar, a.budget);
            if (prof_any) {
              pcs[7] += We - Wd;
              pcs[8] += clock64() - We;
            }
            if (!oke) {
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
    // ------------------------------------------------ selection + solver
    uint8_t* A = smem + p.off_a;
    float* Ls = reinterpret_cast<float*>(smem + p.off_L);       // packed L, [pos][128]
    int* sel = reinterpret_cast<int*>(smem + p.off_sel);        // [m][128]
    float* ys = reinterpret_cast<float*>(smem + p.off_y);       // [m][128]
    float* gs = reinterpret_cast<float*>(smem + p.off_g);       // [m][128]
    float* idg = reinterpret_cast<float*>(smem + p.off_idg);   // [m][128] 1 / L(m, m)
    float* cv = reinterpret_cast<float*>(smem + p.off_cand);    // [128][4][NCAND]
    int* cj = reinterpret_cast<int*>(smem + p.off_cand + TILE_M * 4 * NCAND * 4);
    float* sig = reinterpret_cast<float*>(smem + p.off_sig);
    float* rsm = reinterpret_cast<float*>(smem + p.off_r);  // [12][512] residual slices
    if constexpr (PREC == 2) {
      for (int j = tid; j < p.Kp; j += NEPI) sig[j] = a.sigma[j];
      // FP8 rows hold 64 bytes: bytes 48..63 are zero padding, written once
      for (int row = tid; row < TILE_M; row += NEPI)
        *reinterpret_cast<uint4*>(A + 3 * TILE_M * 16 + row * 16) = make_uint4(0, 0, 0, 0);
    }
    const int R1 = 32 * (warp & 3) + lane, q1 = warp >> 2;
    const int R2 = 8 * warp + (lane >> 2), u = lane & 3;
    const uint32_t trow = tmem_base + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                          static_cast<uint32_t>(q1 * QC);
#define LS(rr, cc2) Ls[(((rr) * ((rr) + 1)) / 2 + (cc2)) * TILE_M + R2]
#define IDG(rr) idg[(rr) * TILE_M + R2]
    long long cc = 0;
    bool ok = true;
    const bool prof_on = prof_any && tid == 0;
    // pre: this tile's signals were written into the A operand (and the MMA
    // warp released) during the previous tile's last iteration; pre_rn2 is
    // the thread's row's ||x||^2 from then
    bool pre = false;
    float pre_rn2 = 0.f;
    // FP16 parts: the inverse scale of the staged operand's correlations (the
    // tile being encoded / the next tile, staged early)
    float cur_rinv = 1.f, pre_rinv = 1.f;
    // Writes the sub-lane's 12 dims of row R2 of tile `tl` into A (FP8 scaled
    // by the row's max; FP16 parts by a power of two) and returns the row's
    // ||x||^2; rinv: the inverse of the correlations' scale (FP16 parts)
    auto stage_x = [&](int tl, bool to_rsm, float& rinv) -> float {
      const int64_t tg0 = static_cast<int64_t>(tl) * TILE_M;
      const bool tin = R2 < (NS - tg0 < TILE_M ? NS - tg0 : TILE_M);
      const float* txr = a.X + (tg0 + R2) * DLSH_D + 12 * u;
      float x[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) x[k] = (tin && 12 * u + k < DLSH_D) ? __ldg(txr + k) : 0.f;
      float part = 0.f;
#pragma unroll
      for (int k = 0; k < 12; ++k) part = fmaf(x[k], x[k], part);
      float inv = 1.f;
      if constexpr (PREC == 2) {
        float mx = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) mx = fmaxf(mx, fabsf(x[k]));
        mx = quad_max(mx);
        inv = mx > 0.f ? FP8_MAX / mx : 1.f;
      }
      if constexpr (PREC == OPF16X2) inv = f16_scale(x, rinv);
      write_a_part<PREC>(A, R2, u, x, inv);
      if constexpr (RESCORE) {
        if (to_rsm) {
#pragma unroll
          for (int k = 0; k < 12; ++k) rsm[k * NEPI + tid] = x[k];
        }
      }
      return quad_sum(part);
    };
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int s = p.s, K = p.K, nchunks = p.nchunks;
      const float eps2 = a.eps * a.eps;
      const int64_t g0 = static_cast<int64_t>(tile) * TILE_M;
      const int rows = static_cast<int>(NS - g0 < TILE_M ? NS - g0 : TILE_M);
      // -------- each sub-lane loads its 12 dims of the signal (a warp reads 8
      // consecutive rows: one contiguous 1440-byte span)
      // x and r live in registers only during the solver phase (the selection
      // phase needs the registers); x is re-read from L1/L2, r kept in smem.
      const float* xr = a.X + (g0 + R2) * DLSH_D + 12 * u;
      const bool in_tile = R2 < rows;
      auto load_x = [&](float (&x)[12]) {
#pragma unroll
        for (int k = 0; k < 12; ++k) x[k] = (in_tile && 12 * u + k < DLSH_D) ? __ldg(xr + k) : 0.f;
      };
      float xnorm, rn2;
      bool active = in_tile;
      int t = 0;
      if (!pre) {
        rn2 = stage_x(tile, true, cur_rinv);
        fence_proxy_async_smem();
        named_bar_sync(1, NEPI);
        if (tid == 0) mbar_arrive(bar_a);
      } else {
        rn2 = pre_rn2;
        cur_rinv = pre_rinv;
        if constexpr (RESCORE) {
          // the residual copy starts as x (rsm was in use until the last barrier)
          float x[12];
          load_x(x);
#pragma unroll
          for (int k = 0; k < 12; ++k) rsm[k * NEPI + tid] = x[k];
        }
      }
      xnorm = sqrtf(rn2);
      pre = false;

      for (int it = 0; it < s; ++it) {
        const long long T0 = prof_on ? clock64() : 0;
        // ================= phase 1: selection over this thread's column quarter
        auto acquire = [&](long long ccq) -> bool {  // wait for the chunk's MMAs
          const int buf = static_cast<int>(ccq % NBUF);
          const long long W0 = prof_on ? clock64() : 0;
          if (!mbar_wait(&bar_full[buf], static_cast<uint32_t>((ccq / NBUF) & 1), a.budget)) {
            flag_status(a.status, ST_TIMEOUT);
            return false;
          }
          if (prof_on) pcs[0] += clock64() - W0;
          tc_fence_after();
          return true;
        };
        auto release = [&](long long ccq) {  // the chunk's TMEM buffer may be reused
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bar_empty[static_cast<int>(ccq % NBUF)]);
        };
        {
          // Argmax of |c| on 32-bit keys: |c| with its low 5 mantissa bits
          // replaced by 31 - k (k = column within the quarter), so one integer
          // max per element yields the largest value and, among values equal
          // to 2^-18 relative, the smallest column.  Chunks are compared on
          // the value bits only (strictly greater wins), so ties go to the
          // smallest atom index overall.  FP32: this is the selection.  BF16 and
          // FP8: each thread's winner (one per column quarter) is a candidate
          // that the solver re-scores in FP32.  Atoms already in the support
          // are not masked here (see the solver's stop rule).
          uint32_t best = 0;
          int bestc = 0;
          // top-4 keys: |c| truncated to its bits above ib, then the column
          // within the quarter (chunk * 32 + k) as (2^ib - 1) - column, so
          // larger keys are larger values and, among equal truncated values,
          // smaller columns
          const uint32_t vmask = 0x7fffffffu & ~((1u << p.ib) - 1u);
          uint32_t run[4] = {0u, 0u, 0u, 0u};
          for (int c = 0; c < nchunks; ++c, ++cc) {
            if (!acquire(cc)) {
              ok = false;
              break;
            }
            __syncwarp();
            uint32_t rr[QC];
            tmem_ld_issue<QC>(trow + static_cast<uint32_t>((cc % NBUF) * BN), rr);
            tmem_ld_wait<QC>(rr);
            release(cc);
            if constexpr (PREC == 2) {
              const int j0 = c * BN + q1 * QC;
#pragma unroll
              for (int k = 0; k < QC; ++k) rr[k] = __float_as_uint(__uint_as_float(rr[k]) * sig[j0 + k]);
            }
            if constexpr (T4) {
              static_assert(QC == 32, "top-4 keys pack a 5-bit column in the chunk");
#pragma unroll
              for (int k = 0; k < QC; ++k) rr[k] = (rr[k] & vmask) | static_cast<uint32_t>(31 - k);
              uint32_t ct[4];
              top4_of8(rr, ct);
#pragma unroll
              for (int o = 8; o < QC; o += 8) {
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
              for (int k = 0; k < QC; k += 2) {
                m0 = max(m0, (rr[k] & 0x7fffffe0u) | static_cast<uint32_t>(31 - k));
                m1 = max(m1, (rr[k + 1] & 0x7fffffe0u) | static_cast<uint32_t>(30 - k));
              }
              const uint32_t m = max(m0, m1);
              if ((m & ~31u) > (best & ~31u)) {
                best = m;
                bestc = c;
              }
            }
          }
          if constexpr (T4) {
            uint32_t* ck = reinterpret_cast<uint32_t*>(smem + p.off_cand) + (R1 * 4 + q1) * 4;
#pragma unroll
            for (int i = 0; i < 4; ++i) ck[i] = run[i];
          } else {
            cv[R1 * 4 + q1] = __uint_as_float(best & ~31u);
            cj[R1 * 4 + q1] = bestc * BN + q1 * QC + 31 - static_cast<int>(best & 31u);
          }
        }
        const long long T1 = prof_on ? clock64() : 0;
        // barrier + vote: every selection thread leaves together if any wait ran out
        if (named_bar_or(1, NEPI, !ok)) {
          ok = false;
          break;
        }
        // Last iteration: every chunk has been read, so the A operand is free.
        // Stage the next tile's signals now and release the MMA warp, so the
        // next tile's first correlations run during this solver phase.
        if (it + 1 == s && tile + static_cast<int>(gridDim.x) < ntiles) {
          pre_rn2 = stage_x(tile + static_cast<int>(gridDim.x), false, pre_rinv);
          fence_proxy_async_smem();
          named_bar_sync(1, NEPI);
          if (tid == 0) mbar_arrive(bar_a);
          pre = true;
        }
        const long long T2 = prof_on ? clock64() : 0;

        // ================= phase 2: merge, re-score, Cholesky, solve, residual
        // Per-iteration quantities live in registers (arrays of t entries, the
        // step compiled once per t); the factor L, y, gamma and the support
        // stay in shared memory across iterations.
        if (active && rn2 <= eps2) active = false;
        if (active) {
          float x[12], r[12];
          load_x(x);
          if constexpr (RESCORE) {
#pragma unroll
            for (int k = 0; k < 12; ++k) r[k] = rsm[k * NEPI + tid];
          }
          int sl[SMAX];
#pragma unroll
          for (int m = 0; m < SMAX; ++m) sl[m] = m < t ? sel[m * TILE_M + R2] : 0;
          int js = -1;
          float best = -1.f;
          if constexpr (EXACT) {
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const float v = cv[R2 * 4 + qq];
              const int j = cj[R2 * 4 + qq];
              if (j < K && (v > best || (v == best && j < js))) {
                best = v;
                js = j;
              }
            }
            // Support atoms are not masked in phase 1: the residual is
            // orthogonal to them, so their |c| sits at rounding level and one
            // of them wins only when every atom's correlation is at that
            // level.  The row then stops, as no atom can reduce the residual
            // by more than rounding.
            bool dup = false;
#pragma unroll
            for (int m = 0; m < SMAX; ++m) dup |= (m < t && sl[m] == js);
            if (dup) js = -1;
          } else {
            // the candidates re-scored in FP32: c = r . d_j.  T4: the row's
            // exact low-precision top 4, merged from the four quarters' top-4
            // lists (sub-lane u reads quarter u, two butterfly rounds) on
            // 64-bit keys (truncated |c|, then the smaller atom index);
            // otherwise the four column-quarter winners.
            int cjr[4];
            if constexpr (T4) {
              const uint32_t* ck = reinterpret_cast<const uint32_t*>(smem + p.off_cand) + (R2 * 4 + u) * 4;
              const uint32_t imask = (1u << p.ib) - 1u;
              const uint32_t vmask = 0x7fffffffu & ~imask;
              unsigned long long lst[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const uint32_t key = ck[i];
                const uint32_t col = imask - (key & imask);
                const uint32_t j = (col >> 5) * BN + static_cast<uint32_t>(u * QC) + (col & 31u);
                lst[i] = key == 0u ? 0ull
                                   : (static_cast<unsigned long long>(key & vmask) << 32) |
                                         static_cast<unsigned long long>(0xFFFFFFFFu - j);
              }
#pragma unroll
              for (int o = 1; o <= 2; o <<= 1) {
                unsigned long long oth[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) oth[i] = __shfl_xor_sync(quad_mask(), lst[i], o);
                merge_top4(lst, oth);
              }
#pragma unroll
              for (int i = 0; i < 4; ++i)
                cjr[i] = lst[i] == 0ull ? 0x7fffffff
                                        : static_cast<int>(0xFFFFFFFFu - static_cast<uint32_t>(lst[i]));
            } else {
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) cjr[qq] = cj[R2 * 4 + qq];
            }
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const int j = cjr[qq];
              float c0 = 0.f;
              if (j < K) {
                const float4* dr = reinterpret_cast<const float4*>(a.D32p + static_cast<size_t>(j) * DPAD + 12 * u);
#pragma unroll
                for (int w4 = 0; w4 < 3; ++w4) {
                  const float4 dv = __ldg(dr + w4);
                  c0 = fmaf(r[4 * w4 + 0], dv.x, c0);
                  c0 = fmaf(r[4 * w4 + 1], dv.y, c0);
                  c0 = fmaf(r[4 * w4 + 2], dv.z, c0);
                  c0 = fmaf(r[4 * w4 + 3], dv.w, c0);
                }
              }
              c0 = fabsf(quad_sum(c0));
              if (j < K && (c0 > best || (c0 == best && j < js))) {
                best = c0;
                js = j;
              }
            }
          }
          if constexpr (RESCORE) {
            bool dup = false;
#pragma unroll
            for (int m = 0; m < SMAX; ++m) dup |= (m < t && sl[m] == js);
            if (dup) js = -1;  // only support atoms were left: every |c| at rounding level
          }
          if (js < 0 || !(best * cur_rinv > CORR_STOP_REL * xnorm)) {
            active = false;
          } else {
            auto step = [&](auto tag) {
              constexpr int T = decltype(tag)::value;
              constexpr int TA = T > 0 ? T : 1;
              // -------- Gram row entries of the support and the new atom's
              // dictionary row
              const float* Grow = a.G + static_cast<size_t>(js) * K;
              float gv[TA];
#pragma unroll
              for (int m = 0; m < T; ++m) gv[m] = __ldg(Grow + sl[m]);
              const float gjj = __ldg(Grow + js);
              float4 dj[3];
              {
                const float4* dr = reinterpret_cast<const float4*>(a.D32p + static_cast<size_t>(js) * DPAD + 12 * u);
#pragma unroll
                for (int w4 = 0; w4 < 3; ++w4) dj[w4] = __ldg(dr + w4);
              }
              // -------- Cholesky update: w = L^-1 g, g_m = <d_js, d_sel[m]>
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
              for (int m = 0; m < T; ++m) LS(T, m) = w[m];  // the four sub-lanes store identical values
              LS(T, T) = ell;
              IDG(T) = iell;
              float bp = 0.f;
#pragma unroll
              for (int w4 = 0; w4 < 3; ++w4) {
                bp = fmaf(dj[w4].x, x[4 * w4 + 0], bp);
                bp = fmaf(dj[w4].y, x[4 * w4 + 1], bp);
                bp = fmaf(dj[w4].z, x[4 * w4 + 2], bp);
                bp = fmaf(dj[w4].w, x[4 * w4 + 3], bp);
              }
              // the 16-atom instantiation reads y and the new factor row w back
              // from shared memory where they are used, instead of holding
              // them in registers across the back substitution (spills)
              constexpr bool REG = SMAX <= 8;
              float yv[REG ? TA : 1];
              if constexpr (REG) {
#pragma unroll
                for (int m = 0; m < T; ++m) yv[m] = ys[m * TILE_M + R2];
              }
              auto y_at = [&](int m) -> float {
                if constexpr (REG) return yv[m];
                else return ys[m * TILE_M + R2];
              };
              auto w_at = [&](int m) -> float {
                if constexpr (REG) return w[m];
                else return LS(T, m);
              };
              float yt = quad_sum(bp);
#pragma unroll
              for (int m = 0; m < T; ++m) yt = fmaf(-w_at(m), y_at(m), yt);
              yt *= iell;
              ys[T * TILE_M + R2] = yt;
              sel[T * TILE_M + R2] = js;
              // back substitution L^T gamma = y (the new atom's entry first)
              const float gt = yt * iell;
              float gam[TA];
#pragma unroll
              for (int m = T - 1; m >= 0; --m) {
                float acc = y_at(m);
#pragma unroll
                for (int q = m + 1; q < T; ++q) acc = fmaf(-LS(q, m), gam[q], acc);
                acc = fmaf(-w_at(m), gt, acc);
                gam[m] = acc * IDG(m);
              }
#pragma unroll
              for (int m = 0; m < T; ++m) gs[m * TILE_M + R2] = gam[m];
              gs[T * TILE_M + R2] = gt;
              // residual r = x - D_I gamma on this sub-lane's 12 dims
#pragma unroll
              for (int k = 0; k < 12; ++k) r[k] = x[k];
              // the support atoms' rows in groups of up to 4, all loads of a
              // group issued before its FMAs (one L2 round trip per group)
#pragma unroll
              for (int m0 = 0; m0 < T; m0 += 4) {
                float4 dv[4][3];
#pragma unroll
                for (int mm = 0; mm < 4; ++mm)
                  if (m0 + mm < T) {
                    const float4* da =
                        reinterpret_cast<const float4*>(a.D32p + static_cast<size_t>(sl[m0 + mm]) * DPAD + 12 * u);
#pragma unroll
                    for (int w4 = 0; w4 < 3; ++w4) dv[mm][w4] = __ldg(da + w4);
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
              t = T + 1;
              float pr = 0.f;
#pragma unroll
              for (int k = 0; k < 12; ++k) pr = fmaf(r[k], r[k], pr);
              rn2 = quad_sum(pr);
              if (it + 1 < s) {
                float inv = 1.f;
                if constexpr (PREC == 2) {
                  float mx = 0.f;
#pragma unroll
                  for (int k = 0; k < 12; ++k) mx = fmaxf(mx, fabsf(r[k]));
                  mx = quad_max(mx);
                  inv = mx > 0.f ? FP8_MAX / mx : 1.f;
                }
                if constexpr (PREC == OPF16X2) inv = f16_scale(r, cur_rinv);
                write_a_part<PREC>(A, R2, u, r, inv);
              }
              if constexpr (RESCORE) {
#pragma unroll
                for (int k = 0; k < 12; ++k) rsm[k * NEPI + tid] = r[k];
              }
            };
            if (t < SMAX)
              with_t<SMAX>(t, step);
            else
              active = false;
          }
        }
        fence_proxy_async_smem();
        const long long T3 = prof_on ? clock64() : 0;
        named_bar_sync(1, NEPI);
        if (it + 1 < s && tid == 0) mbar_arrive(bar_a);
        const long long Tend = prof_on ? clock64() : 0;
        if (prof_on) {
          pcs[1] += T1 - T0;
          pcs[2] += T2 - T1;
          pcs[3] += T3 - T2;
          pcs[4] += Tend - T3;
          pcs[5] += 1;
        }
      }
      if (!ok) break;
      if (R2 < rows) {
        const int64_t g = g0 + R2;
        for (int mm = u; mm < s; mm += 4) {
          a.idx[g * s + mm] = mm < t ? static_cast<uint16_t>(sel[mm * TILE_M + R2]) : static_cast<uint16_t>(0);
          a.coef[g * s + mm] = mm < t ? gs[mm * TILE_M + R2] : 0.f;
        }
        if (u == 0) {
          a.nnz[g] = static_cast<uint8_t>(t);
          if (a.resid_sq) a.resid_sq[g] = rn2;
        }
      }
    }
#undef LS
#undef IDG
  }
  tc_fence_before();
  __syncthreads();
  if (prof_any && tid == 0) {
    for (int k = 0; k < 10; ++k) atomicAdd(a.prof + k, pcs[k]);
    if (blockIdx.x == 0) a.prof[11] = 1;  // the variant that ran: one tile per CTA
  }
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}

#include "encode_pair.cuh"
#include "encode_alt.cuh"
#include "encode_split.cuh"

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

template <int PREC, int BN, bool T4 = false>
static int launch_encode(const Args& a, int grid, cudaStream_t st) {
  auto fn = a.p.s <= 8 ? encode_kernel<PREC, BN, 8, T4> : encode_kernel<PREC, BN, 16, T4>;
  DLSH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT),
                "dlsh_encode: cudaFuncSetAttribute");
  fn<<<grid, NTHREADS, a.p.smem, st>>>(a);
  count_launches(1);
  return check_launch("dlsh_encode: launch");
}

template <int PREC, bool T4>
static int launch_pair(const PairArgs& a, int grid, cudaStream_t st) {
  auto fn = encode_pair_kernel<PREC, T4>;
  DLSH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT),
                "dlsh_encode: cudaFuncSetAttribute");
  fn<<<grid, NTHREADS, a.p.smem, st>>>(a);
  count_launches(1);
  return check_launch("dlsh_encode: launch");
}

static int launch_alt(const AltArgs& a, int grid, cudaStream_t st) {
  DLSH_CUDA_TRY(cudaFuncSetAttribute(encode_alt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SMEM_LIMIT),
                "dlsh_encode: cudaFuncSetAttribute");
  encode_alt_kernel<<<grid, NTHREADS, a.p.smem, st>>>(a);
  count_launches(1);
  return check_launch("dlsh_encode: launch");
}

template <bool F16, int NS>
static int launch_split(const SplitArgs& a, int grid, cudaStream_t st) {
  DLSH_CUDA_TRY(cudaFuncSetAttribute(encode_split_kernel<F16, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SMEM_LIMIT),
                "dlsh_encode: cudaFuncSetAttribute");
  encode_split_kernel<F16, NS><<<grid, NTHREADS, a.p.smem, st>>>(a);
  count_launches(1);
  return check_launch("dlsh_encode: launch");
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
