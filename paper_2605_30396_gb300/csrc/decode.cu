// Radiance straight from the sparse codes (Sec. 2.2): the renderer's SH step
// reads the shared dictionary and each Gaussian's nonzeros instead of its 45 SH
// coefficients.  For Gaussian i and unit view direction v_i,
//   rgb_c = sum_b Y_b(v_i) * sum_{t < nnz_i} coef[i,t] * D[idx[i,t], c*15 + b].
//
// Memory-bound design: the FP32 dictionary is staged once per CTA in shared
// memory and every nonzero costs three 16-lane reads of one dictionary row.  A
// warp works on batches of 16 Gaussians: first all of the batch's codes are
// loaded (coalesced) into shared memory while one lane per Gaussian computes its
// direction and 15 basis values; then each half-warp takes one Gaussian, lane b
// owning basis b of all three channels, accumulates sum_t coef * D[j_t, c*15+b],
// multiplies by Y_b and reduces across the half with shuffles.  Results are
// staged and written back coalesced.
#include <cuda_fp16.h>
#include <math.h>

#include "common.cuh"
#include "host.hpp"
#include "sh.cuh"

namespace dlsh {
namespace dec {

constexpr int ROW = 45;         // dictionary row in shared memory (plus 16 zero words at the end)
constexpr int YS = 17;          // basis values per Gaussian slot (15 used, slot 15 holds nnz)
constexpr int SMEM_LIMIT = 232448;

// Per-warp shared memory: basis slots, staged rgb, and the batch's codes.
constexpr int GB = 16;          // Gaussians per warp batch (small batches: more warps fit per SM)
__host__ __device__ constexpr int warp_floats(int s) { return GB * YS + GB * 3 + GB * s * 2; }

__constant__ ShConst g_sh;

template <bool SMEM_D>
__global__ void __launch_bounds__(1024) decode_kernel(
    const float* __restrict__ D, int K, const uint16_t* __restrict__ idx,
    const float* __restrict__ coef, const uint8_t* __restrict__ nnz, int s, int64_t N,
    const float* __restrict__ dm, int use_cam, float cx, float cy, float cz,
    float* __restrict__ rgb, uint32_t* status) {
  extern __shared__ __align__(16) float sm[];
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* Ds = sm;
  const int dwords = SMEM_D ? K * ROW + 16 : 0;
  float* wsm = sm + dwords + warp * warp_floats(s);
  float* Ys = wsm;
  float* outs = wsm + GB * YS;
  float* ccoef = outs + GB * 3;
  uint32_t* cidx = reinterpret_cast<uint32_t*>(ccoef + GB * s);
  if (SMEM_D) {
    for (int f = threadIdx.x; f < dwords; f += blockDim.x) Ds[f] = f < K * ROW ? D[f] : 0.f;
    __syncthreads();
  }
  const int hl = lane & 15, h = lane >> 4;
  const unsigned FULL = 0xffffffffu;
  const int64_t nbatch = (N + GB - 1) / GB;
  const int64_t wstride = static_cast<int64_t>(gridDim.x) * nwarps;
  bool bad = false;
  for (int64_t bt = static_cast<int64_t>(blockIdx.x) * nwarps + warp; bt < nbatch; bt += wstride) {
    const int64_t base = bt * GB;
    const int nb = N - base < GB ? static_cast<int>(N - base) : GB;
    // ---- phase A: every load of the batch is issued here, then one lane per
    // Gaussian computes its direction and 15 basis values
    for (int f = lane; f < nb * s; f += 32) {
      cidx[f] = idx[base * s + f];
      ccoef[f] = coef[base * s + f];
    }
    {
      const int64_t g = base + lane;
      float vx = 0.f, vy = 0.f, vz = 1.f;
      int nz = 0;
      if (lane < nb) {
        vx = dm[g * 3 + 0];
        vy = dm[g * 3 + 1];
        vz = dm[g * 3 + 2];
        nz = nnz[g];
        if (use_cam) {
          vx -= cx;
          vy -= cy;
          vz -= cz;
          const float inv = rsqrtf(vx * vx + vy * vy + vz * vz);
          vx *= inv;
          vy *= inv;
          vz *= inv;
        }
      }
      float Y[15];
      sh_basis(g_sh.c, vx, vy, vz, Y);
      if (lane < GB) {
#pragma unroll
        for (int q = 0; q < 15; ++q) Ys[lane * YS + q] = Y[q];
        Ys[lane * YS + 15] = __int_as_float(nz);
      }
    }
    __syncwarp();
    // ---- phase B: a half-warp per Gaussian, lane hl owns basis hl of R, G, B
    for (int pp = 0; pp < GB / 2; ++pp) {
      const int gl = 2 * pp + h;
      int nz = gl < nb ? __float_as_int(Ys[gl * YS + 15]) : 0;
      if (nz > s) {
        bad = true;
        nz = s;
      }
      float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
      for (int t = 0; t < s; ++t) {
        uint32_t j = 0;
        float a = 0.f;
        if (t < nz) {
          j = cidx[gl * s + t];
          a = ccoef[gl * s + t];
        }
        if (j >= static_cast<uint32_t>(K)) {
          bad = true;
          j = 0;
          a = 0.f;
        }
        if (SMEM_D) {
          const float* row = Ds + j * ROW + hl;
          acc0 = fmaf(a, row[0], acc0);
          acc1 = fmaf(a, row[15], acc1);
          acc2 = fmaf(a, row[30], acc2);
        } else if (hl < 15) {
          const float* row = D + static_cast<size_t>(j) * DLSH_D + hl;
          acc0 = fmaf(a, __ldg(row), acc0);
          acc1 = fmaf(a, __ldg(row + 15), acc1);
          acc2 = fmaf(a, __ldg(row + 30), acc2);
        }
      }
      // lane 15 read a neighbouring word (finite) times Y = 0
      const float yb = hl < 15 ? Ys[gl * YS + hl] : 0.f;
      float p0 = acc0 * yb, p1 = acc1 * yb, p2 = acc2 * yb;
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) {
        p0 += __shfl_xor_sync(FULL, p0, off);
        p1 += __shfl_xor_sync(FULL, p1, off);
        p2 += __shfl_xor_sync(FULL, p2, off);
      }
      if (hl == 0) {
        outs[gl * 3 + 0] = p0;
        outs[gl * 3 + 1] = p1;
        outs[gl * 3 + 2] = p2;
      }
    }
    __syncwarp();
    // ---- coalesced store of the batch's outputs
#pragma unroll
    for (int q = 0; q < (GB * 3 + 31) / 32; ++q) {
      const int e = lane + 32 * q;
      if (e < nb * 3) rgb[base * 3 + e] = outs[e];
    }
    __syncwarp();
  }
  if (bad) flag_status(status, ST_BAD_INPUT);
}

// ---- compact storage: FP16 coefficients, 8- or 16-bit atom indices ----------
// The dictionary is staged in shared memory as FP16, 16 slots of four halves
// per atom (slot b < 15: the R, G, B coefficients of basis b, then a zero):
// 128 bytes per atom, so a half-warp reads one atom's row for all three
// channels in a single 8-byte load per lane (one wavefront), where the FP32
// kernel needs three.  Sums stay FP32.
template <int IDXB>
__global__ void __launch_bounds__(1024) decode_compact_kernel(
    const float* __restrict__ D, int K, const void* __restrict__ idxv,
    const __half* __restrict__ coef, const uint8_t* __restrict__ nnz, int s, int64_t N,
    const float* __restrict__ dm, int use_cam, float cx, float cy, float cz,
    float* __restrict__ rgb, uint32_t* status) {
  extern __shared__ __align__(16) float sm[];
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint2* Ds = reinterpret_cast<uint2*>(sm);  // [K][16]
  float* wsm = sm + static_cast<size_t>(K) * 32 + warp * warp_floats(s);
  float* Ys = wsm;
  float* outs = wsm + GB * YS;
  float* ccoef = outs + GB * 3;
  uint32_t* cidx = reinterpret_cast<uint32_t*>(ccoef + GB * s);
  for (int f = threadIdx.x; f < K * 16; f += blockDim.x) {
    const int j = f >> 4, b = f & 15;
    uint2 v = make_uint2(0u, 0u);
    if (b < 15) {
      const float* dr = D + static_cast<size_t>(j) * DLSH_D + b;
      const __half2 rg = __floats2half2_rn(dr[0], dr[15]);
      const __half2 bz = __floats2half2_rn(dr[30], 0.f);
      v.x = *reinterpret_cast<const uint32_t*>(&rg);
      v.y = *reinterpret_cast<const uint32_t*>(&bz);
    }
    Ds[f] = v;
  }
  __syncthreads();
  const int hl = lane & 15, h = lane >> 4;
  const unsigned FULL = 0xffffffffu;
  const int64_t nbatch = (N + GB - 1) / GB;
  const int64_t wstride = static_cast<int64_t>(gridDim.x) * nwarps;
  bool bad = false;
  for (int64_t bt = static_cast<int64_t>(blockIdx.x) * nwarps + warp; bt < nbatch; bt += wstride) {
    const int64_t base = bt * GB;
    const int nb = N - base < GB ? static_cast<int>(N - base) : GB;
    for (int f = lane; f < nb * s; f += 32) {
      cidx[f] = IDXB == 1 ? static_cast<uint32_t>(static_cast<const uint8_t*>(idxv)[base * s + f])
                          : static_cast<uint32_t>(static_cast<const uint16_t*>(idxv)[base * s + f]);
      ccoef[f] = __half2float(coef[base * s + f]);
    }
    {
      const int64_t g = base + lane;
      float vx = 0.f, vy = 0.f, vz = 1.f;
      int nz = 0;
      if (lane < nb) {
        vx = dm[g * 3 + 0];
        vy = dm[g * 3 + 1];
        vz = dm[g * 3 + 2];
        nz = nnz[g];
        if (use_cam) {
          vx -= cx;
          vy -= cy;
          vz -= cz;
          const float inv = rsqrtf(vx * vx + vy * vy + vz * vz);
          vx *= inv;
          vy *= inv;
          vz *= inv;
        }
      }
      float Y[15];
      sh_basis(g_sh.c, vx, vy, vz, Y);
      if (lane < GB) {
#pragma unroll
        for (int q = 0; q < 15; ++q) Ys[lane * YS + q] = Y[q];
        Ys[lane * YS + 15] = __int_as_float(nz);
      }
    }
    __syncwarp();
    for (int pp = 0; pp < GB / 2; ++pp) {
      const int gl = 2 * pp + h;
      int nz = gl < nb ? __float_as_int(Ys[gl * YS + 15]) : 0;
      if (nz > s) {
        bad = true;
        nz = s;
      }
      float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
      for (int t = 0; t < s; ++t) {
        uint32_t j = 0;
        float a = 0.f;
        if (t < nz) {
          j = cidx[gl * s + t];
          a = ccoef[gl * s + t];
        }
        if (j >= static_cast<uint32_t>(K)) {
          bad = true;
          j = 0;
          a = 0.f;
        }
        const uint2 v = Ds[j * 16 + hl];
        const float2 rg = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
        const float2 bz = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
        acc0 = fmaf(a, rg.x, acc0);
        acc1 = fmaf(a, rg.y, acc1);
        acc2 = fmaf(a, bz.x, acc2);
      }
      const float yb = hl < 15 ? Ys[gl * YS + hl] : 0.f;
      float p0 = acc0 * yb, p1 = acc1 * yb, p2 = acc2 * yb;
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) {
        p0 += __shfl_xor_sync(FULL, p0, off);
        p1 += __shfl_xor_sync(FULL, p1, off);
        p2 += __shfl_xor_sync(FULL, p2, off);
      }
      if (hl == 0) {
        outs[gl * 3 + 0] = p0;
        outs[gl * 3 + 1] = p1;
        outs[gl * 3 + 2] = p2;
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < (GB * 3 + 31) / 32; ++q) {
      const int e = lane + 32 * q;
      if (e < nb * 3) rgb[base * 3 + e] = outs[e];
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

static int upload_constants(cudaStream_t st) {
  static thread_local int uploaded_dev = -1;
  int dev = 0;
  DLSH_CUDA_TRY(cudaGetDevice(&dev), "dlsh_decode: cudaGetDevice");
  if (uploaded_dev == dev) return DLSH_OK;
  const ShConst k = make_sh_constants();
  DLSH_CUDA_TRY(cudaMemcpyToSymbolAsync(g_sh, &k, sizeof(k), 0, cudaMemcpyHostToDevice, st),
                "dlsh_decode: constants");
  DLSH_CUDA_TRY(cudaStreamSynchronize(st), "dlsh_decode: constants");
  uploaded_dev = dev;
  return DLSH_OK;
}

}  // namespace dec

// Shared with the bench / learn paths: enqueue one decode.
int decode_enqueue(const float* D, int K, const uint16_t* idx, const float* coef,
                   const uint8_t* nnz, int s, int64_t N, const float* dm, const float* cam,
                   float* rgb, uint32_t* status, cudaStream_t st) {
  using namespace dec;
  int rc = upload_constants(st);
  if (rc) return rc;
  if (N == 0) return DLSH_OK;
  int sms = device_sm_count();
  if (sms <= 0) sms = 1;
  const float cx = cam ? cam[0] : 0.f, cy = cam ? cam[1] : 0.f, cz = cam ? cam[2] : 0.f;
  const int64_t nbatch = (N + GB - 1) / GB;
  const size_t dbytes = (static_cast<size_t>(K) * ROW + 16) * 4;
  const size_t wbytes = static_cast<size_t>(warp_floats(s)) * 4;
  int nwarps = static_cast<int>((SMEM_LIMIT - static_cast<long long>(dbytes)) / static_cast<long long>(wbytes));
  if (nwarps > 32) nwarps = 32;
  if (nwarps >= 6) {
    const size_t smem = dbytes + static_cast<size_t>(nwarps) * wbytes;
    DLSH_CUDA_TRY(cudaFuncSetAttribute(decode_kernel<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT),
                  "dlsh_decode: attribute");
    int per_sm = static_cast<int>(SMEM_LIMIT / smem);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = static_cast<int64_t>(sms) * per_sm;
    const int64_t need = (nbatch + nwarps - 1) / nwarps;
    if (grid > need) grid = need;
    decode_kernel<true><<<static_cast<int>(grid), nwarps * 32, smem, st>>>(
        D, K, idx, coef, nnz, s, N, dm, cam != nullptr, cx, cy, cz, rgb, status);
  } else {
    const int nw = 8;
    const size_t smem = static_cast<size_t>(nw) * wbytes;
    DLSH_CUDA_TRY(cudaFuncSetAttribute(decode_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT),
                  "dlsh_decode: attribute");
    int64_t grid = static_cast<int64_t>(sms) * 4;
    const int64_t need = (nbatch + nw - 1) / nw;
    if (grid > need) grid = need;
    decode_kernel<false><<<static_cast<int>(grid), nw * 32, smem, st>>>(
        D, K, idx, coef, nnz, s, N, dm, cam != nullptr, cx, cy, cz, rgb, status);
  }
  count_launches(1);
  return check_launch("dlsh_decode: launch");
}

}  // namespace dlsh

extern "C" int dlsh_decode(const float* D, int K, int d, const uint16_t* idx, const float* coef,
                           const uint8_t* nnz, int s, int64_t N, const float* dirs_or_means,
                           const float* cam_pos, float* rgb, void* stream, int flags) {
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
  int rc = decode_enqueue(D, K, idx, coef, nnz, s, N, dirs_or_means, cam_pos, rgb, nullptr, st);
  if (rc) return rc;
  return finish(st, nullptr, flags, "dlsh_decode");
}

namespace dlsh {
namespace dec {
inline size_t compact_dict_bytes(int K) { return static_cast<size_t>(K) * 128; }
}  // namespace dec
}  // namespace dlsh

extern "C" size_t dlsh_decode_compact_max_k(int s) {
  using namespace dlsh::dec;
  if (s < 1 || s > DLSH_MAX_S) return 0;
  const size_t wb = static_cast<size_t>(warp_floats(s)) * 4;
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
                                   const float* dirs_or_means, const float* cam_pos, float* rgb,
                                   void* stream, int flags) {
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
    int sms = device_sm_count();
    if (sms <= 0) sms = 1;
    const float cx = cam_pos ? cam_pos[0] : 0.f, cy = cam_pos ? cam_pos[1] : 0.f,
                cz = cam_pos ? cam_pos[2] : 0.f;
    const int64_t nbatch = (N + GB - 1) / GB;
    const size_t dbytes = compact_dict_bytes(K);
    const size_t wbytes = static_cast<size_t>(warp_floats(s)) * 4;
    int nwarps = static_cast<int>((SMEM_LIMIT - static_cast<long long>(dbytes)) / static_cast<long long>(wbytes));
    if (nwarps > 32) nwarps = 32;
    const size_t smem = dbytes + static_cast<size_t>(nwarps) * wbytes;
    int per_sm = static_cast<int>(SMEM_LIMIT / smem);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = static_cast<int64_t>(sms) * per_sm;
    const int64_t need = (nbatch + nwarps - 1) / nwarps;
    if (grid > need) grid = need;
    const __half* cf = reinterpret_cast<const __half*>(coef_f16);
    if (idx_bytes == 1) {
      DLSH_CUDA_TRY(cudaFuncSetAttribute(decode_compact_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_LIMIT),
                    "dlsh_decode_compact: attribute");
      decode_compact_kernel<1><<<static_cast<int>(grid), nwarps * 32, smem, st>>>(
          D, K, idx, cf, nnz, s, N, dirs_or_means, cam_pos != nullptr, cx, cy, cz, rgb, nullptr);
    } else {
      DLSH_CUDA_TRY(cudaFuncSetAttribute(decode_compact_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_LIMIT),
                    "dlsh_decode_compact: attribute");
      decode_compact_kernel<2><<<static_cast<int>(grid), nwarps * 32, smem, st>>>(
          D, K, idx, cf, nnz, s, N, dirs_or_means, cam_pos != nullptr, cx, cy, cz, rgb, nullptr);
    }
    count_launches(1);
    rc = check_launch("dlsh_decode_compact: launch");
    if (rc) return rc;
  }
  return finish(st, nullptr, flags, "dlsh_decode_compact");
}
