// Radiance straight from the sparse codes (Sec. 2.2): the renderer's SH step
// reads the shared dictionary and each Gaussian's nonzeros instead of its 45 SH
// coefficients.  For Gaussian i and unit view direction v_i,
//   rgb_c = sum_b Y_b(v_i) * sum_{t < nnz_i} coef[i,t] * D[idx[i,t], c*15 + b].
//
// Bound by shared-memory wavefronts, not HBM: the dictionary is staged once
// per CTA in shared memory and every nonzero reads a whole atom (45 values).
// A warp takes batches of 8 (FP32 table) or 16 Gaussians: the batch's codes are loaded
// (coalesced) into shared memory as (index, coefficient) pairs while one lane
// per Gaussian computes its direction and 15 basis values; then eight lanes take
// one Gaussian (four Gaussians per warp step) and read contiguous spans of the
// atom:
//  - FP32 table: three channel planes of 16 floats per atom (192 bytes); lane
//    q reads 16 bytes of the R and G planes (lanes 0-3: R of bases 4q..4q+3,
//    lanes 4-7: G), one 128-byte span per Gaussian, and 8 bytes of the B plane
//    (bases 2q, 2q+1); the channel sums are reduced in five shuffles;
//  - FP16 table (compact storage): 16 slots of (R, G, B, 0) halves per atom
//    (128 bytes), lane q reading bases 2q and 2q+1 of all three channels in
//    one 16-byte word; its three channel sums are reduced over the eight lanes
//    in four shuffles (a transposing butterfly).
// Results are staged and written back coalesced.  For dictionaries too large
// for shared memory the FP32 rows are read through the read-only cache, with
// the FP16 path's lane mapping.
#include <cuda_fp16.h>
#include <math.h>
#include <stdio.h>

#include "common.cuh"
#include "host.hpp"
#include "sh.cuh"

namespace dlsh {
namespace dec {

enum : int { FM_F32 = 0, FM_GLOBAL = 1, FM_C8 = 2, FM_C16 = 3 };

constexpr int YS = 16;          // basis values per Gaussian slot (15 and a zero)
// A slot is four 16-byte words; word k of slot g sits at word k ^ ((g >> 1) & 3),
// so that the slot writes of a batch (one lane per Gaussian, 16-byte stores)
// fall on different bank groups.  Returns the float offset of word k.
__device__ __forceinline__ int ysw(int g, int k) { return (k ^ ((g >> 1) & 3)) * 4; }
constexpr int SMEM_LIMIT = 232448;
// Gaussians per warp batch by default: 8 beside the 192 KB FP32 table (small
// batches let more warps fit in the shared memory left), 16 with the FP16 table
// (whose warps already reach 32 per CTA, where the larger batch costs less per
// Gaussian).  dlsh_autotune_decode may record the other size (8 or 16) and a
// warp count per (format, K, s).
__host__ __device__ constexpr int batch_of(int fm) { return fm == 0 ? 8 : 16; }

// Code slots staged per Gaussian: even (16-byte pair reads), and not a multiple
// of four, so that the four Gaussians of a step read different bank groups.
inline int staged_slots(int s) {
  int sp = (s + 1) & ~1;
  if (sp % 4 == 0) sp += 2;
  return sp;
}
// Per-warp shared memory: basis slots, staged rgb, codes, nnz.
__host__ __device__ constexpr int warp_floats(int sp, int gb) { return gb * YS + gb * 3 + gb * sp * 2 + gb; }
__host__ __device__ constexpr int dict_floats(int fm, int K) { return fm == FM_F32 ? K * 48 : fm >= FM_C8 ? K * 32 : 0; }

__constant__ ShConst g_sh;

template <int FM, int GB>
__global__ void __launch_bounds__(1024) decode_kernel(
    const float* __restrict__ D, int K, const void* __restrict__ idxv, const void* __restrict__ coefv,
    const uint8_t* __restrict__ nnz, int s, int sp, uint32_t sdiv, int64_t N,
    const float* __restrict__ dm, int use_cam, float cx, float cy, float cz,
    const float* __restrict__ dc, float y00, float* __restrict__ rgb, uint32_t* status) {
  extern __shared__ __align__(16) float sm[];
  static_assert(GB == 8 || GB == 16, "batches of 8 or 16 Gaussians");
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  // ---- dictionary in shared memory; four slots per thread per round, their
  // loads issued before any is stored
  const int dwords = dict_floats(FM, K);
  if (FM != FM_GLOBAL) {
    for (int f0 = threadIdx.x; f0 < K * 16; f0 += 4 * blockDim.x) {
      float v[4][3];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int f = f0 + u * blockDim.x, j = f >> 4, b = f & 15;
        const bool live = f < K * 16 && b < 15;
        const float* dr = D + static_cast<size_t>(live ? j : 0) * DLSH_D + (live ? b : 0);
        v[u][0] = live ? dr[0] : 0.f;
        v[u][1] = live ? dr[15] : 0.f;
        v[u][2] = live ? dr[30] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int f = f0 + u * blockDim.x;
        if (f >= K * 16) break;
        if (FM == FM_F32) {
          const int j = f >> 4, b = f & 15;
          sm[j * 48 + b] = v[u][0];
          sm[j * 48 + 16 + b] = v[u][1];
          sm[j * 48 + 32 + b] = v[u][2];
        } else {
          const __half2 rg = __floats2half2_rn(v[u][0], v[u][1]);
          const __half2 bz = __floats2half2_rn(v[u][2], 0.f);
          reinterpret_cast<uint2*>(sm)[f] =
              make_uint2(*reinterpret_cast<const uint32_t*>(&rg), *reinterpret_cast<const uint32_t*>(&bz));
        }
      }
    }
    __syncthreads();
  }
  float* wsm = sm + dwords + warp * warp_floats(sp, GB);
  float* Ys = wsm;
  float* outs = wsm + GB * YS;
  uint2* cpk = reinterpret_cast<uint2*>(wsm + GB * YS + GB * 3);
  int* nzs = reinterpret_cast<int*>(wsm + GB * YS + GB * 3 + GB * sp * 2);
  const int ql = lane & 7, grp = lane >> 3;
  const int64_t nbatch = (N + GB - 1) / GB;
  const int64_t wstride = static_cast<int64_t>(gridDim.x) * nwarps;
  bool bad = false;
  for (int64_t bt = static_cast<int64_t>(blockIdx.x) * nwarps + warp; bt < nbatch; bt += wstride) {
    const int64_t base = bt * GB;
    const int nb = N - base < GB ? static_cast<int>(N - base) : GB;
    // direction inputs first: their loads are in flight while the codes are staged
    const int64_t g = base + lane;
    float vx = 0.f, vy = 0.f, vz = 1.f;
    int nz = 0;
    if (lane < nb) {
      vx = dm[g * 3 + 0];
      vy = dm[g * 3 + 1];
      vz = dm[g * 3 + 2];
      nz = nnz[g];
    }
    // ---- phase A: the batch's codes as (index, coefficient) pairs, element
    // f = lane + 32 k (k < s/2 rounded up), four loads in flight per lane
    for (int k0 = 0; 32 * k0 < GB * s; k0 += 4) {
      uint32_t jj[4];
      float aa[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int f = lane + 32 * (k0 + u);
        jj[u] = 0;
        aa[u] = 0.f;
        if (f < nb * s) {
          const int64_t e = base * s + f;
          if (FM == FM_F32 || FM == FM_GLOBAL) {
            jj[u] = static_cast<const uint16_t*>(idxv)[e];
            aa[u] = static_cast<const float*>(coefv)[e];
          } else {
            jj[u] = FM == FM_C8 ? static_cast<uint32_t>(static_cast<const uint8_t*>(idxv)[e])
                                : static_cast<uint32_t>(static_cast<const uint16_t*>(idxv)[e]);
            aa[u] = __half2float(static_cast<const __half*>(coefv)[e]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int f = lane + 32 * (k0 + u);
        if (f < nb * s) {
          const int gl = s == 1 ? f : static_cast<int>(__umulhi(static_cast<uint32_t>(f), sdiv));
          // an index beyond the dictionary is reported and counts as zero
          const bool ok = jj[u] < static_cast<uint32_t>(K);
          bad |= !ok;
          cpk[gl * sp + (f - gl * s)] = make_uint2(ok ? jj[u] : 0u, ok ? __float_as_uint(aa[u]) : 0u);
        }
      }
    }
    if (lane < GB)
      for (int t = s; t < sp; ++t) cpk[lane * sp + t] = make_uint2(0u, 0u);
    {
      if (use_cam && lane < nb) {
        vx -= cx;
        vy -= cy;
        vz -= cz;
        const float inv = rsqrtf(vx * vx + vy * vy + vz * vz);
        vx *= inv;
        vy *= inv;
        vz *= inv;
      }
      float Y[15];
      sh_basis(g_sh.c, vx, vy, vz, Y);
      if (lane < GB) {
        float* ys = Ys + lane * YS;
        *reinterpret_cast<float4*>(ys + ysw(lane, 0)) = make_float4(Y[0], Y[1], Y[2], Y[3]);
        *reinterpret_cast<float4*>(ys + ysw(lane, 1)) = make_float4(Y[4], Y[5], Y[6], Y[7]);
        *reinterpret_cast<float4*>(ys + ysw(lane, 2)) = make_float4(Y[8], Y[9], Y[10], Y[11]);
        *reinterpret_cast<float4*>(ys + ysw(lane, 3)) = make_float4(Y[12], Y[13], Y[14], 0.f);
        if (nz > s) {
          bad = true;
          nz = s;
        }
        nzs[lane] = nz;
      }
      __syncwarp();  // the batch's codes are staged
      // entries t >= nnz count as zero: clear them, so that the loop below
      // needs no per-entry test
      if (lane < GB)
        for (int t = nz; t < s; ++t) cpk[lane * sp + t] = make_uint2(0u, 0u);
    }
    __syncwarp();
    // ---- phase B: eight lanes per Gaussian, four Gaussians per step
    for (int g0 = 0; g0 < nb; g0 += 4) {
      const int gl = g0 + grp;
      const bool act = gl < nb;
      const int gs = act ? gl : 0;
      const int nzl = act ? nzs[gs] : 0;
      int nzp = max(nzl, __shfl_xor_sync(FULL, nzl, 8));
      nzp = max(nzp, __shfl_xor_sync(FULL, nzp, 16));
      if (FM == FM_F32) {
        // FP32 planes: lane ql reads 16 bytes of the R and G planes (lanes
        // 0-3: R of bases 4ql..4ql+3; lanes 4-7: G of bases 4(ql-4)..), so the
        // eight lanes of a Gaussian read one contiguous 128-byte span, and
        // 8 bytes of the B plane (bases 2ql, 2ql+1)
        float4 acc4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 accb = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int t = 0; t < nzp; t += 2) {
          const uint4 c2 = *reinterpret_cast<const uint4*>(cpk + gs * sp + t);
          const uint32_t jt[2] = {c2.x, c2.z};
          const float at[2] = {__uint_as_float(c2.y), __uint_as_float(c2.w)};
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const float a = at[u];
            const float* row = sm + jt[u] * 48;
            const float4 w = *reinterpret_cast<const float4*>(row + 4 * ql);
            const float2 bb = *reinterpret_cast<const float2*>(row + 32 + 2 * ql);
            acc4.x = fmaf(a, w.x, acc4.x);
            acc4.y = fmaf(a, w.y, acc4.y);
            acc4.z = fmaf(a, w.z, acc4.z);
            acc4.w = fmaf(a, w.w, acc4.w);
            accb.x = fmaf(a, bb.x, accb.x);
            accb.y = fmaf(a, bb.y, accb.y);
          }
        }
        const float4 y4 = *reinterpret_cast<const float4*>(Ys + gs * YS + ysw(gs, ql & 3));
        const float2 yb = *reinterpret_cast<const float2*>(Ys + gs * YS + ysw(gs, ql >> 1) + ((2 * ql) & 3));
        float prg = fmaf(y4.x, acc4.x, fmaf(y4.y, acc4.y, fmaf(y4.z, acc4.z, y4.w * acc4.w)));
        float pb = fmaf(yb.x, accb.x, yb.y * accb.y);
        // R over lanes 0-3, G over lanes 4-7, B over all eight
        prg += __shfl_xor_sync(FULL, prg, 1);
        prg += __shfl_xor_sync(FULL, prg, 2);
        pb += __shfl_xor_sync(FULL, pb, 1);
        pb += __shfl_xor_sync(FULL, pb, 2);
        pb += __shfl_xor_sync(FULL, pb, 4);
        if (act && ql == 0) {
          outs[gl * 3 + 0] = prg;
          outs[gl * 3 + 2] = pb;
        }
        if (act && ql == 4) outs[gl * 3 + 1] = prg;
        continue;
      }
      float aR = 0.f, aG = 0.f, aB = 0.f, bR = 0.f, bG = 0.f, bBl = 0.f;
#pragma unroll 2
      for (int t = 0; t < nzp; t += 2) {
        const uint4 c2 = *reinterpret_cast<const uint4*>(cpk + gs * sp + t);
        const uint32_t jt[2] = {c2.x, c2.z};
        const float at[2] = {__uint_as_float(c2.y), __uint_as_float(c2.w)};
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const float a = at[u];
          if (FM == FM_GLOBAL) {
            // bases 2ql and 2ql + 1 of the atom's row (basis 15 does not exist)
            const float* row = D + static_cast<size_t>(jt[u]) * DLSH_D + 2 * ql;
            aR = fmaf(a, __ldg(row), aR);
            aG = fmaf(a, __ldg(row + 15), aG);
            aB = fmaf(a, __ldg(row + 30), aB);
            if (ql < 7) {
              bR = fmaf(a, __ldg(row + 1), bR);
              bG = fmaf(a, __ldg(row + 16), bG);
              bBl = fmaf(a, __ldg(row + 31), bBl);
            }
          } else {
            const uint4 w = reinterpret_cast<const uint4*>(sm)[jt[u] * 8 + ql];
            const float2 rg = __half22float2(*reinterpret_cast<const __half2*>(&w.x));
            const float2 bz = __half22float2(*reinterpret_cast<const __half2*>(&w.y));
            const float2 rh = __half22float2(*reinterpret_cast<const __half2*>(&w.z));
            const float2 bh = __half22float2(*reinterpret_cast<const __half2*>(&w.w));
            aR = fmaf(a, rg.x, aR);
            aG = fmaf(a, rg.y, aG);
            aB = fmaf(a, bz.x, aB);
            bR = fmaf(a, rh.x, bR);
            bG = fmaf(a, rh.y, bG);
            bBl = fmaf(a, bh.x, bBl);
          }
        }
      }
      const float2 yy = *reinterpret_cast<const float2*>(Ys + gs * YS + ysw(gs, ql >> 1) + ((2 * ql) & 3));
      const float p0 = fmaf(yy.x, aR, yy.y * bR), p1 = fmaf(yy.x, aG, yy.y * bG),
                  p2 = fmaf(yy.x, aB, yy.y * bBl);
      // transposing butterfly over the 8 lanes: afterwards lane ql holds
      // channel ql >> 1 (ql = 0, 2, 4)
      const bool b2 = (ql & 4) != 0, b1 = (ql & 2) != 0;
      const float r0 = __shfl_xor_sync(FULL, b2 ? p0 : p2, 4);
      const float r1 = __shfl_xor_sync(FULL, b2 ? p1 : 0.f, 4);
      const float k0 = (b2 ? p2 : p0) + r0;
      const float k1 = (b2 ? 0.f : p1) + r1;
      float m = (b1 ? k1 : k0) + __shfl_xor_sync(FULL, b1 ? k0 : k1, 2);
      m += __shfl_xor_sync(FULL, m, 1);
      if (act && (ql & 1) == 0 && ql < 6) outs[gl * 3 + (ql >> 1)] = m;
    }
    __syncwarp();
    // ---- coalesced store of the batch's outputs
#pragma unroll
    for (int q = 0; q < (GB * 3 + 31) / 32; ++q) {
      const int e = lane + 32 * q;
      if (e < nb * 3) {
        float v = outs[e];
        // full colour: the DC term and the usual +0.5 offset, clamped at zero
        if (dc) v = fmaxf(0.f, fmaf(y00, dc[base * 3 + e], v) + 0.5f);
        rgb[base * 3 + e] = v;
      }
    }
    __syncwarp();
  }
  if (bad) flag_status(status, ST_BAD_INPUT);
}

// ELL codes -> compact codes (round-to-nearest FP16 coefficients, narrowed
// indices); padding slots keep index 0 and coefficient 0.
__global__ void compact_codes_kernel(const uint16_t* __restrict__ idx, const float* __restrict__ coef,
                                     int64_t n, int idx_bytes, void* __restrict__ idx_out,
                                     __half* __restrict__ coef_out) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n) return;
  if (idx_bytes == 1) static_cast<uint8_t*>(idx_out)[e] = static_cast<uint8_t>(idx[e]);
  else static_cast<uint16_t*>(idx_out)[e] = idx[e];
  coef_out[e] = __float2half_rn(coef[e]);
}

// The SH constants go to each device once (the first decode on a device should
// therefore not be inside a stream capture).
static int upload_constants(cudaStream_t st) {
  static PerDevice<int> uploaded;
  int ok = 0;
  return uploaded.get(&ok, [&](int& v) {
    const ShConst k = make_sh_constants();
    DLSH_CUDA_TRY(cudaMemcpyToSymbolAsync(g_sh, &k, sizeof(k), 0, cudaMemcpyHostToDevice, st),
                  "dlsh_decode: constants");
    DLSH_CUDA_TRY(cudaStreamSynchronize(st), "dlsh_decode: constants");
    v = 1;
    return DLSH_OK;
  });
}

// One decode launch with the dictionary format FM: shared-memory sizes from
// the format, as many warps per CTA as shared memory allows (at most 32), and
// a grid of (CTAs resident per SM) x SMs, capped by the work.
template <int FM, int GB>
static int launch_decode_gb(const float* D, int K, const void* idx, const void* coef, const uint8_t* nnz,
                            int s, int64_t N, const float* dm, const float* cam, const float* dc, float* rgb,
                            uint32_t* status, int nwarps, cudaStream_t st, const char* call) {
  int sms = device_sm_count();
  if (sms <= 0) sms = 1;
  const int sp = staged_slots(s);
  const uint32_t sdiv = s >= 2 ? static_cast<uint32_t>((uint64_t(1) << 32) / static_cast<uint64_t>(s) + 1) : 0u;
  constexpr int gb = GB;
  const size_t smem = static_cast<size_t>(dict_floats(FM, K) + nwarps * warp_floats(sp, gb)) * 4;
  DLSH_CUDA_TRY(
      cudaFuncSetAttribute(decode_kernel<FM, GB>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT), call);
  int per_sm = 0;
  DLSH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, decode_kernel<FM, GB>, nwarps * 32, smem),
                call);
  if (per_sm < 1) per_sm = 1;
  const int64_t nbatch = (N + gb - 1) / gb;
  int64_t grid = static_cast<int64_t>(sms) * per_sm;
  const int64_t need = (nbatch + nwarps - 1) / nwarps;
  if (grid > need) grid = need;
  const float cx = cam ? cam[0] : 0.f, cy = cam ? cam[1] : 0.f, cz = cam ? cam[2] : 0.f;
  const float y00 = static_cast<float>(0.5 / sqrt(M_PI));
  decode_kernel<FM, GB><<<static_cast<int>(grid), nwarps * 32, smem, st>>>(
      D, K, idx, coef, nnz, s, sp, sdiv, N, dm, cam != nullptr, cx, cy, cz, dc, y00, rgb, status);
  count_launches(1);
  return check_launch(call);
}

// Warps per CTA that fit beside the dictionary of format fm with batches of gb
// Gaussians (0 if none do).
static int fit_warps(int fm, int K, int s, int gb) {
  const long long room = SMEM_LIMIT - 4LL * dict_floats(fm, K);
  const long long wb = 4LL * warp_floats(staged_slots(s), gb);
  long long n = room > 0 ? room / wb : 0;
  return static_cast<int>(n > 32 ? 32 : n);
}
static int fit_warps(int fm, int K, int s) { return fit_warps(fm, K, s, batch_of(fm)); }

// The batch size and warps per CTA for (fm, K, s): the autotuner's record if it
// still fits, else the default batch with as many warps as fit (16 warps for
// rows read through the read-only cache).
static void decode_shape(int fm, int K, int s, int* gb, int* nw) {
  char key[64];
  snprintf(key, sizeof(key), "decode f=%d K=%d s=%d", fm, K, s);
  int v[2] = {0, 0};
  if (tune_get(key, v, 2) && (v[0] == 8 || v[0] == 16) && v[1] >= 1 &&
      v[1] <= (fm == FM_GLOBAL ? 32 : fit_warps(fm, K, s, v[0]))) {
    *gb = v[0];
    *nw = v[1];
    return;
  }
  *gb = batch_of(fm);
  *nw = fm == FM_GLOBAL ? 16 : fit_warps(fm, K, s);
}

// One decode launch of format FM with a batch of gb Gaussians per warp.
template <int FM>
static int launch_decode(const float* D, int K, const void* idx, const void* coef, const uint8_t* nnz, int s,
                         int64_t N, const float* dm, const float* cam, const float* dc, float* rgb,
                         uint32_t* status, int gb, int nwarps, cudaStream_t st, const char* call) {
  if (gb == 16)
    return launch_decode_gb<FM, 16>(D, K, idx, coef, nnz, s, N, dm, cam, dc, rgb, status, nwarps, st, call);
  return launch_decode_gb<FM, 8>(D, K, idx, coef, nnz, s, N, dm, cam, dc, rgb, status, nwarps, st, call);
}

}  // namespace dec

// The FP32 table stays in shared memory while at least six warps (batches of
// 8) fit beside it; beyond that (about 1150 atoms) the rows are read through
// the read-only cache.
static int decode_format(int K, int s) {
  return dec::fit_warps(dec::FM_F32, K, s) >= 6 ? dec::FM_F32 : dec::FM_GLOBAL;
}

// Shared with the bench / learn paths: enqueue one decode.
int decode_enqueue(const float* D, int K, const uint16_t* idx, const float* coef,
                   const uint8_t* nnz, int s, int64_t N, const float* dm, const float* cam,
                   const float* dc, float* rgb, uint32_t* status, cudaStream_t st) {
  using namespace dec;
  int rc = upload_constants(st);
  if (rc) return rc;
  if (N == 0) return DLSH_OK;
  const int fm = decode_format(K, s);
  int gb = 0, nw = 0;
  decode_shape(fm, K, s, &gb, &nw);
  if (fm == FM_F32)
    return launch_decode<FM_F32>(D, K, idx, coef, nnz, s, N, dm, cam, dc, rgb, status, gb, nw, st, "dlsh_decode");
  return launch_decode<FM_GLOBAL>(D, K, idx, coef, nnz, s, N, dm, cam, dc, rgb, status, gb, nw, st,
                                  "dlsh_decode");
}

}  // namespace dlsh

extern "C" int dlsh_decode(const float* D, int K, int d, const uint16_t* idx, const float* coef,
                           const uint8_t* nnz, int s, int64_t N, const float* dirs_or_means,
                           const float* cam_pos, const float* dc, float* rgb, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  if (d != DLSH_D) return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_decode: d must be 45, got %d", d);
  if (K < 1 || K > DLSH_MAX_K)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_decode: K must be in [1, 65535], got %d", K);
  if (s < 1 || s > DLSH_MAX_S)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_decode: s must be in [1, 32], got %d", s);
  if (N < 0) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_decode: N < 0");
  if (!D) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_decode: D is NULL");
  if (N > 0 && (!idx || !coef || !nnz || !dirs_or_means || !rgb))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_decode: NULL array");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = decode_enqueue(D, K, idx, coef, nnz, s, N, dirs_or_means, cam_pos, dc, rgb, nullptr, st);
  if (rc) return rc;
  return finish(st, nullptr, flags, "dlsh_decode");
}

extern "C" size_t dlsh_decode_compact_max_k(int s) {
  using namespace dlsh::dec;
  if (s < 1 || s > DLSH_MAX_S) return 0;
  const size_t wb = static_cast<size_t>(warp_floats(staged_slots(s), batch_of(FM_C8))) * 4;
  return (static_cast<size_t>(SMEM_LIMIT) - 6 * wb) / 128;
}

extern "C" int dlsh_compact_codes(const uint16_t* idx, const float* coef, int64_t N, int s, int K,
                                  void* idx_out, int idx_bytes, uint16_t* coef_out, void* stream,
                                  int flags) {
  using namespace dlsh;
  clear_error();
  if (N < 0 || s < 1 || s > DLSH_MAX_S || K < 1 || K > DLSH_MAX_K)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_compact_codes: bad sizes");
  if (idx_bytes != 1 && idx_bytes != 2)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_compact_codes: idx_bytes must be 1 or 2");
  if (idx_bytes == 1 && K > 256)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_compact_codes: 8-bit indices need K <= 256, got %d", K);
  if (N > 0 && (!idx || !coef || !idx_out || !coef_out))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_compact_codes: NULL array");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = N * s;
  if (n > 0) {
    dec::compact_codes_kernel<<<static_cast<int>((n + 255) / 256), 256, 0, st>>>(
        idx, coef, n, idx_bytes, idx_out, reinterpret_cast<__half*>(coef_out));
    count_launches(1);
  }
  return finish(st, nullptr, flags, "dlsh_compact_codes");
}

extern "C" int dlsh_decode_compact(const float* D, int K, int d, const void* idx, int idx_bytes,
                                   const uint16_t* coef_f16, const uint8_t* nnz, int s, int64_t N,
                                   const float* dirs_or_means, const float* cam_pos, const float* dc,
                                   float* rgb, void* stream, int flags) {
  using namespace dlsh;
  using namespace dlsh::dec;
  clear_error();
  if (d != DLSH_D) return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_decode_compact: d must be 45, got %d", d);
  if (s < 1 || s > DLSH_MAX_S)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_decode_compact: s must be in [1, 32], got %d", s);
  if (K < 1 || static_cast<size_t>(K) > dlsh_decode_compact_max_k(s))
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_decode_compact: K=%d exceeds the shared-memory dictionary (%zu)",
                     K, dlsh_decode_compact_max_k(s));
  if (idx_bytes != 1 && idx_bytes != 2)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_decode_compact: idx_bytes must be 1 or 2");
  if (idx_bytes == 1 && K > 256)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_decode_compact: 8-bit indices need K <= 256");
  if (N < 0) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_decode_compact: N < 0");
  if (!D) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_decode_compact: D is NULL");
  if (N > 0 && (!idx || !coef_f16 || !nnz || !dirs_or_means || !rgb))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_decode_compact: NULL array");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = upload_constants(st);
  if (rc) return rc;
  if (N > 0) {
    const int fm = idx_bytes == 1 ? FM_C8 : FM_C16;
    int gb = 0, nw = 0;
    decode_shape(fm, K, s, &gb, &nw);
    rc = fm == FM_C8 ? launch_decode<FM_C8>(D, K, idx, coef_f16, nnz, s, N, dirs_or_means, cam_pos, dc, rgb,
                                            nullptr, gb, nw, st, "dlsh_decode_compact")
                     : launch_decode<FM_C16>(D, K, idx, coef_f16, nnz, s, N, dirs_or_means, cam_pos, dc, rgb,
                                             nullptr, gb, nw, st, "dlsh_decode_compact");
    if (rc) return rc;
  }
  return finish(st, nullptr, flags, "dlsh_decode_compact");
}

extern "C" int dlsh_tuned_decode(int format, int K, int s, int* batch, int* warps) {
  using namespace dlsh;
  using namespace dlsh::dec;
  if (format < 0 || format > 2 || K < 1 || K > DLSH_MAX_K || s < 1 || s > DLSH_MAX_S) return 0;
  const int fm = format == 0 ? decode_format(K, s) : (format == 1 ? FM_C8 : FM_C16);
  char key[64];
  snprintf(key, sizeof(key), "decode f=%d K=%d s=%d", fm, K, s);
  int v[2] = {0, 0};
  if (!tune_get(key, v, 2)) return 0;
  if (batch) *batch = v[0];
  if (warps) *warps = v[1];
  return 1;
}

extern "C" int dlsh_autotune_decode(const float* D, int K, int d, const void* idx, const void* coef, int format,
                                    const uint8_t* nnz, int s, int64_t N, const float* dirs_or_means,
                                    const float* cam_pos, float* rgb, void* stream, int* best_batch,
                                    int* best_warps) {
  using namespace dlsh;
  using namespace dlsh::dec;
  clear_error();
  if (d != DLSH_D) return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_autotune_decode: d must be 45, got %d", d);
  if (format < 0 || format > 2)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_autotune_decode: format must be 0, 1 or 2, got %d", format);
  if (s < 1 || s > DLSH_MAX_S)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_autotune_decode: s must be in [1, 32], got %d", s);
  if (K < 1 || K > DLSH_MAX_K || (format > 0 && static_cast<size_t>(K) > dlsh_decode_compact_max_k(s)) ||
      (format == 1 && K > 256))
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_autotune_decode: K=%d is out of range for format %d", K, format);
  if (N < 1 || !D || !idx || !coef || !nnz || !dirs_or_means || !rgb)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_autotune_decode: need a non-empty sample");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = upload_constants(st);
  if (rc) return rc;
  const int fm = format == 0 ? decode_format(K, s) : (format == 1 ? FM_C8 : FM_C16);
  const char* call = "dlsh_autotune_decode";
  auto run = [&](int gb, int nw) -> int {
    switch (fm) {
      case FM_F32:
        return launch_decode<FM_F32>(D, K, idx, coef, nnz, s, N, dirs_or_means, cam_pos, nullptr, rgb, nullptr, gb,
                                     nw, st, call);
      case FM_GLOBAL:
        return launch_decode<FM_GLOBAL>(D, K, idx, coef, nnz, s, N, dirs_or_means, cam_pos, nullptr, rgb, nullptr,
                                        gb, nw, st, call);
      case FM_C8:
        return launch_decode<FM_C8>(D, K, idx, coef, nnz, s, N, dirs_or_means, cam_pos, nullptr, rgb, nullptr, gb,
                                    nw, st, call);
      default:
        return launch_decode<FM_C16>(D, K, idx, coef, nnz, s, N, dirs_or_means, cam_pos, nullptr, rgb, nullptr,
                                     gb, nw, st, call);
    }
  };
  cudaEvent_t e0, e1;
  DLSH_CUDA_TRY(cudaEventCreate(&e0), "dlsh_autotune_decode: event");
  DLSH_CUDA_TRY(cudaEventCreate(&e1), "dlsh_autotune_decode: event");
  int best_gb = 0, best_nw = 0;
  float best_ms = 0.f;
  for (int gb : {8, 16}) {
    // as many warps as fit beside the dictionary, three quarters and half of that
    const int maxw = fm == FM_GLOBAL ? 32 : fit_warps(fm, K, s, gb);
    int cand[3], nc = 0;
    for (int w : {maxw, maxw * 3 / 4, maxw / 2}) {
      bool seen = false;
      for (int i = 0; i < nc; ++i) seen |= cand[i] == w;
      if (w >= 1 && !seen) cand[nc++] = w;
    }
    for (int i = 0; i < nc && !rc; ++i) {
      float sum = 0.f;
      for (int rep = 0; rep < 4 && !rc; ++rep) {
        cudaEventRecord(e0, st);
        rc = run(gb, cand[i]);
        cudaEventRecord(e1, st);
        if (rc) break;
        const cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
          rc = cuda_fail(e, "dlsh_autotune_decode: event");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) sum += ms;  // the first run warms up
      }
      if (!rc && (best_gb == 0 || sum < best_ms)) {
        best_gb = gb;
        best_nw = cand[i];
        best_ms = sum;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (best_gb == 0) return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_autotune_decode: no shape fits");
  char key[64];
  snprintf(key, sizeof(key), "decode f=%d K=%d s=%d", fm, K, s);
  const int v[2] = {best_gb, best_nw};
  tune_put(key, v, 2);
  if (best_batch) *best_batch = best_gb;
  if (best_warps) *best_warps = best_nw;
  return finish(st, nullptr, 0, call);
}
