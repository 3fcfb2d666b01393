// The encoder's kernels and the device code they share.  The host side is in
// encode.cu; the kernels are instantiated in enc_one_fp32.cu, enc_one_lowp.cu,
// enc_pair.cu and enc_split.cu (each with the launch wrappers of its family),
// so that the families compile in parallel.
//
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
#pragma once

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
inline int make_plan(int K, int s, int code, Plan& p, int bn = 0, int smem_limit = SMEM_LIMIT,
                     bool f16 = false) {
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

template <int PREC, int BN, bool T4 = false>
int launch_encode(const Args& a, int grid, cudaStream_t st) {
  auto fn = a.p.s <= 8 ? encode_kernel<PREC, BN, 8, T4> : encode_kernel<PREC, BN, 16, T4>;
  DLSH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT),
                "dlsh_encode: cudaFuncSetAttribute");
  fn<<<grid, NTHREADS, a.p.smem, st>>>(a);
  count_launches(1);
  return check_launch("dlsh_encode: launch");
}

template <int PREC, bool T4>
int launch_pair(const PairArgs& a, int grid, cudaStream_t st) {
  auto fn = encode_pair_kernel<PREC, T4>;
  DLSH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT),
                "dlsh_encode: cudaFuncSetAttribute");
  fn<<<grid, NTHREADS, a.p.smem, st>>>(a);
  count_launches(1);
  return check_launch("dlsh_encode: launch");
}

// One launch of the alternating two-tile encoder (defined in enc_split.cu).
int launch_alt(const AltArgs& a, int grid, cudaStream_t st);

template <bool F16, int NS>
int launch_split(const SplitArgs& a, int grid, cudaStream_t st) {
  DLSH_CUDA_TRY(cudaFuncSetAttribute(encode_split_kernel<F16, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SMEM_LIMIT),
                "dlsh_encode: cudaFuncSetAttribute");
  encode_split_kernel<F16, NS><<<grid, NTHREADS, a.p.smem, st>>>(a);
  count_launches(1);
  return check_launch("dlsh_encode: launch");
}

// Explicitly instantiated in enc_one_fp32.cu, enc_one_lowp.cu, enc_pair.cu and
// enc_split.cu, so that each kernel family is compiled in one translation unit.
extern template int launch_encode<0, 64, false>(const Args&, int, cudaStream_t);
extern template int launch_encode<0, 128, false>(const Args&, int, cudaStream_t);
extern template int launch_encode<OPF16X2, 128, false>(const Args&, int, cudaStream_t);
extern template int launch_encode<1, 128, false>(const Args&, int, cudaStream_t);
extern template int launch_encode<1, 128, true>(const Args&, int, cudaStream_t);
extern template int launch_encode<2, 128, false>(const Args&, int, cudaStream_t);
extern template int launch_encode<2, 128, true>(const Args&, int, cudaStream_t);
extern template int launch_pair<0, false>(const PairArgs&, int, cudaStream_t);
extern template int launch_pair<1, false>(const PairArgs&, int, cudaStream_t);
extern template int launch_pair<1, true>(const PairArgs&, int, cudaStream_t);
extern template int launch_pair<2, false>(const PairArgs&, int, cudaStream_t);
extern template int launch_pair<2, true>(const PairArgs&, int, cudaStream_t);
extern template int launch_split<false, 2>(const SplitArgs&, int, cudaStream_t);
extern template int launch_split<true, 2>(const SplitArgs&, int, cudaStream_t);
extern template int launch_split<true, 3>(const SplitArgs&, int, cudaStream_t);

}  // namespace enc
}  // namespace dlsh
