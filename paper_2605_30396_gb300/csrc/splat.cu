// Splatting preprocess with the colour step read from the sparse codes
// (Sec. 2.2): per Gaussian, project the mean and the 3D covariance to the
// screen, cull, and evaluate the view-dependent colour either from the 45 dense
// SH coefficients (the baseline renderer) or from the shared dictionary and the
// Gaussian's nonzeros (the paper's renderer).  Both variants do the same
// geometry; they differ only in where the colour coefficients come from.
//
// Geometry (the usual splatting forms; p_c = R mu + t):
//   Sigma    = R(q) diag(s)^2 R(q)^T,  q = (w, x, y, z) normalised
//   J        = [[fx/z, 0, -fx x'/z], [0, fy/z, -fy y'/z]],  x' = clamp(x/z, +-1.3 W/(2 fx))
//   Sigma2D  = (J R) Sigma (J R)^T + 0.3 I
//   conic    = Sigma2D^-1,  radius = ceil(3 sqrt(lambda_max)),
//   lambda_max = mid + sqrt(max(0.1, mid^2 - det)),  mid = trace / 2
//   visible  = z > z_near, det > 0, and the radius square meets the image
//   rgb      = max(0, Y00 dc + sum_b Y_b(v) y_{c,b} + 0.5),  v = (mu - cam) / |mu - cam|
// Culled Gaussians get radius 0 and zeros elsewhere, and their colour
// coefficients are never read.
//
// A warp takes 32 Gaussians at a time.  Phase A: one lane per Gaussian does the
// geometry and the 15 basis values and the warp ballots the visible ones.
// Phase B (colour):
//  - dense SH: the visible Gaussians' 180-byte rows are copied (cp.async,
//    4-byte granules, coalesced along each row) into a per-warp stage, and each
//    lane then dots its own row (stride 45 words: no bank conflicts) with its
//    basis values;
//  - codes: the dictionary sits in shared memory as 16 slots of (R, G, B, 0)
//    per atom, FP32 (256 bytes) or FP16 (128 bytes); the batch's codes are
//    staged as (index, coefficient) pairs, and eight lanes take one visible
//    Gaussian, each lane owning two bases of the three channels; the channel
//    sums are reduced over the eight lanes in four shuffles (a transposing
//    butterfly).
#include <cuda_fp16.h>
#include <math.h>

#include "common.cuh"
#include "host.hpp"
#include "sh.cuh"

namespace dlsh {
namespace spl {

enum : int { CM_SH = 0, CM_F32 = 1, CM_C8 = 2, CM_C16 = 3 };

constexpr int GB = 32;         // Gaussians per warp batch
constexpr int ROW = 45;        // dense SH row
constexpr int YS = 16;         // basis slot per Gaussian (15 values and a zero)
constexpr int SMEM_LIMIT = 232448;
constexpr float kLowpass = 0.3f;
constexpr float kClamp = 1.3f;

struct Params {
  const float* means;
  const float* scales;
  const float4* quats;
  const float* dc;
  const float* sh;       // CM_SH: [N x 45]
  const float* D;        // codes: [K x 45] FP32
  const void* idx;       // codes: [N x s] u16 (CM_F32, CM_C16) or u8 (CM_C8)
  const void* coef;      // codes: [N x s] FP32 (CM_F32) or FP16 bits
  const uint8_t* nnz;    // codes: [N]
  float2* xy;
  float* depth;
  float* conic;
  int* radius;
  float* rgb;
  int64_t N;
  int K, s, sp;          // sp: staged code slots per Gaussian (even)
  int sh_aligned;        // dense SH rows start on a 16-byte boundary
  uint32_t sdiv;         // floor(2^32 / s) + 1 (s >= 2): f / s = umulhi(f, sdiv) for f < 2^16
  float R[9], t[3];
  float fx, fy, W, H, hw, hh, limx, limy, z_near;
  float cam[3];          // camera centre -R^T t
  float y00;             // 1 / (2 sqrt(pi))
  float shc[15];
};

__host__ __device__ constexpr int dense_warp_floats() { return GB * ROW + GB; }
__host__ __device__ constexpr int codes_warp_floats(int sp) { return GB * YS + GB * 3 + GB * sp * 2 + 2 * GB; }
// shared-memory dictionary: 16 slots per atom (basis b < 15, then zeros) of
// (R, G, B, 0) as FP32 (256 bytes) or FP16 (128 bytes)
__host__ __device__ constexpr int dict_floats(int cm, int K) { return cm == 1 ? K * 64 : cm >= 2 ? K * 32 : 0; }

inline int staged_slots(int s) {
  int sp = (s + 1) & ~1;
  if (sp % 4 == 0) sp += 2;  // two halves' 16-byte code reads fall in different bank groups
  return sp;
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// a0 b0 + a1 b1 + a2 b2, rounded in a fixed order
__device__ __forceinline__ float dot3(float a0, float a1, float a2, float b0, float b1, float b2) {
  return fmaf(a0, b0, fmaf(a1, b1, __fmul_rn(a2, b2)));
}

template <int CM>
__global__ void __launch_bounds__(1024) preprocess_kernel(const __grid_constant__ Params p) {
  extern __shared__ __align__(16) float sm[];
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const int K = p.K, s = p.s, sp = p.sp;

  // ---- dictionary in shared memory (codes variants); four slots per thread
  // per round, their loads issued before any is converted
  const int dwords = dict_floats(CM, K);
  if (CM != CM_SH) {
    for (int f0 = threadIdx.x; f0 < K * 16; f0 += 4 * blockDim.x) {
      float v[4][3];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int f = f0 + u * blockDim.x, j = f >> 4, b = f & 15;
        const bool live = f < K * 16 && b < 15;
        const float* dr = p.D + static_cast<size_t>(live ? j : 0) * DLSH_D + (live ? b : 0);
        v[u][0] = live ? dr[0] : 0.f;
        v[u][1] = live ? dr[15] : 0.f;
        v[u][2] = live ? dr[30] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int f = f0 + u * blockDim.x;
        if (f >= K * 16) break;
        if (CM == CM_F32) {
          reinterpret_cast<float4*>(sm)[f] = make_float4(v[u][0], v[u][1], v[u][2], 0.f);
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

  float* wsm = sm + dwords + warp * (CM == CM_SH ? dense_warp_floats() : codes_warp_floats(sp));
  // dense: stage [32 x 45], vlist[32]
  // codes: Ys [32 x 16], outs [32 x 3], codes [32 x sp] uint2, vlist[32], nzs[32]
  float* stage = wsm;
  float* Ys = wsm;
  float* outs = wsm + GB * YS;
  uint2* cpk = reinterpret_cast<uint2*>(wsm + GB * YS + GB * 3);
  int* vlist = reinterpret_cast<int*>(CM == CM_SH ? wsm + GB * ROW : wsm + GB * YS + GB * 3 + GB * sp * 2);
  int* nzs = vlist + GB;

  // phase B of the codes variants: a quarter-warp (8 lanes) per Gaussian
  const int ql = lane & 7, grp = lane >> 3;
  const int64_t N = p.N;
  const int64_t nbatch = (N + GB - 1) / GB;
  const int64_t wstride = static_cast<int64_t>(gridDim.x) * nwarps;
  for (int64_t bt = static_cast<int64_t>(blockIdx.x) * nwarps + warp; bt < nbatch; bt += wstride) {
    const int64_t base = bt * GB;
    const int nb = N - base < GB ? static_cast<int>(N - base) : GB;
    const int64_t g = base + lane;
    const bool valid = lane < nb;

    // ---- phase A: geometry, one lane per Gaussian.  Its loads are issued
    // first, so that they are in flight while the codes are staged.
    float mx = 0.f, my = 0.f, mz = 0.f, sx = 0.f, sy = 0.f, sz = 0.f, dr = 0.f, dg = 0.f, db = 0.f;
    float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
    int nz = 0;
    if (valid) {
      mx = p.means[g * 3 + 0];
      my = p.means[g * 3 + 1];
      mz = p.means[g * 3 + 2];
      sx = p.scales[g * 3 + 0];
      sy = p.scales[g * 3 + 1];
      sz = p.scales[g * 3 + 2];
      q = p.quats[g];
      dr = p.dc[g * 3 + 0];
      dg = p.dc[g * 3 + 1];
      db = p.dc[g * 3 + 2];
      if (CM != CM_SH) nz = p.nnz[g];
    }
    // codes of the whole batch, staged as (index, coefficient bits) pairs
    if (CM != CM_SH) {
      // element f = lane + 32 k of the batch (k < s); four loads in flight per lane
      for (int k0 = 0; k0 < s; k0 += 4) {
        uint32_t jj[4];
        float aa[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int f = lane + 32 * (k0 + u);
          jj[u] = 0;
          aa[u] = 0.f;
          if (k0 + u < s && f < nb * s) {
            const int64_t e = base * s + f;
            if (CM == CM_F32) {
              jj[u] = static_cast<const uint16_t*>(p.idx)[e];
              aa[u] = static_cast<const float*>(p.coef)[e];
            } else {
              jj[u] = CM == CM_C8 ? static_cast<uint32_t>(static_cast<const uint8_t*>(p.idx)[e])
                                  : static_cast<uint32_t>(static_cast<const uint16_t*>(p.idx)[e]);
              aa[u] = __half2float(static_cast<const __half*>(p.coef)[e]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int f = lane + 32 * (k0 + u);
          if (k0 + u < s && f < nb * s) {
            const int gl = s == 1 ? f : static_cast<int>(__umulhi(static_cast<uint32_t>(f), p.sdiv));
            // an index beyond the dictionary counts as a zero entry
            const bool ok = jj[u] < static_cast<uint32_t>(K);
            cpk[gl * sp + (f - gl * s)] = make_uint2(ok ? jj[u] : 0u, ok ? __float_as_uint(aa[u]) : 0u);
          }
        }
      }
      for (int t = s; t < sp; ++t) cpk[lane * sp + t] = make_uint2(0u, 0u);
    }

    const float* R = p.R;
    const float x = fmaf(R[0], mx, fmaf(R[1], my, fmaf(R[2], mz, p.t[0])));
    const float y = fmaf(R[3], mx, fmaf(R[4], my, fmaf(R[5], mz, p.t[1])));
    const float z = fmaf(R[6], mx, fmaf(R[7], my, fmaf(R[8], mz, p.t[2])));
    const bool front = valid && z > p.z_near;
    const float zs = front ? z : 1.f;
    const float xs = front ? x : 0.f, ys = front ? y : 0.f;
    // Every product and sum below is rounded explicitly (no contraction left to
    // the compiler), so the geometry is bit-identical whichever colour source
    // the kernel is instantiated for.
    const float iz = __frcp_rn(zs);
    // rotation of the normalised quaternion
    const float qn = rsqrtf(fmaf(q.x, q.x, fmaf(q.y, q.y, fmaf(q.z, q.z, __fmul_rn(q.w, q.w)))));
    const float qw = __fmul_rn(q.x, qn), qx = __fmul_rn(q.y, qn), qy = __fmul_rn(q.z, qn), qz = __fmul_rn(q.w, qn);
    const float r00 = __fsub_rn(1.f, __fmul_rn(2.f, fmaf(qy, qy, __fmul_rn(qz, qz))));
    const float r11 = __fsub_rn(1.f, __fmul_rn(2.f, fmaf(qx, qx, __fmul_rn(qz, qz))));
    const float r22 = __fsub_rn(1.f, __fmul_rn(2.f, fmaf(qx, qx, __fmul_rn(qy, qy))));
    const float r01 = __fmul_rn(2.f, fmaf(qx, qy, -__fmul_rn(qw, qz)));
    const float r02 = __fmul_rn(2.f, fmaf(qx, qz, __fmul_rn(qw, qy)));
    const float r10 = __fmul_rn(2.f, fmaf(qx, qy, __fmul_rn(qw, qz)));
    const float r12 = __fmul_rn(2.f, fmaf(qy, qz, -__fmul_rn(qw, qx)));
    const float r20 = __fmul_rn(2.f, fmaf(qx, qz, -__fmul_rn(qw, qy)));
    const float r21 = __fmul_rn(2.f, fmaf(qy, qz, __fmul_rn(qw, qx)));
    // M = R(q) diag(s); Sigma = M M^T
    const float m00 = __fmul_rn(r00, sx), m01 = __fmul_rn(r01, sy), m02 = __fmul_rn(r02, sz);
    const float m10 = __fmul_rn(r10, sx), m11 = __fmul_rn(r11, sy), m12 = __fmul_rn(r12, sz);
    const float m20 = __fmul_rn(r20, sx), m21 = __fmul_rn(r21, sy), m22 = __fmul_rn(r22, sz);
    const float S00 = dot3(m00, m01, m02, m00, m01, m02);
    const float S01 = dot3(m00, m01, m02, m10, m11, m12);
    const float S02 = dot3(m00, m01, m02, m20, m21, m22);
    const float S11 = dot3(m10, m11, m12, m10, m11, m12);
    const float S12 = dot3(m10, m11, m12, m20, m21, m22);
    const float S22 = dot3(m20, m21, m22, m20, m21, m22);
    // T = J R (2 x 3)
    const float cx = fminf(fmaxf(__fmul_rn(xs, iz), -p.limx), p.limx);
    const float cy = fminf(fmaxf(__fmul_rn(ys, iz), -p.limy), p.limy);
    const float j00 = __fmul_rn(p.fx, iz), j02 = -__fmul_rn(__fmul_rn(p.fx, cx), iz);
    const float j11 = __fmul_rn(p.fy, iz), j12 = -__fmul_rn(__fmul_rn(p.fy, cy), iz);
    const float t00 = fmaf(j00, R[0], __fmul_rn(j02, R[6])), t01 = fmaf(j00, R[1], __fmul_rn(j02, R[7])),
                t02 = fmaf(j00, R[2], __fmul_rn(j02, R[8]));
    const float t10 = fmaf(j11, R[3], __fmul_rn(j12, R[6])), t11 = fmaf(j11, R[4], __fmul_rn(j12, R[7])),
                t12 = fmaf(j11, R[5], __fmul_rn(j12, R[8]));
    // U = T Sigma; Sigma2D = U T^T
    const float u00 = dot3(t00, t01, t02, S00, S01, S02);
    const float u01 = dot3(t00, t01, t02, S01, S11, S12);
    const float u02 = dot3(t00, t01, t02, S02, S12, S22);
    const float u10 = dot3(t10, t11, t12, S00, S01, S02);
    const float u11 = dot3(t10, t11, t12, S01, S11, S12);
    const float u12 = dot3(t10, t11, t12, S02, S12, S22);
    const float ca = __fadd_rn(dot3(u00, u01, u02, t00, t01, t02), kLowpass);
    const float cb = dot3(u00, u01, u02, t10, t11, t12);
    const float cc = __fadd_rn(dot3(u10, u11, u12, t10, t11, t12), kLowpass);
    const float det = fmaf(ca, cc, -__fmul_rn(cb, cb));
    const bool ok = front && det > 0.f;
    const float mid = __fmul_rn(0.5f, __fadd_rn(ca, cc));
    const float lam = __fadd_rn(mid, __fsqrt_rn(fmaxf(0.1f, fmaf(mid, mid, -det))));
    const float rad = ceilf(__fmul_rn(3.f, __fsqrt_rn(fmaxf(lam, 0.f))));
    const float px = fmaf(__fmul_rn(p.fx, xs), iz, p.hw);
    const float py = fmaf(__fmul_rn(p.fy, ys), iz, p.hh);
    const bool vis = ok && px + rad > 0.f && px - rad < p.W && py + rad > 0.f && py - rad < p.H;
    if (valid) {
      const float idet = vis ? __frcp_rn(det) : 0.f;
      p.xy[g] = vis ? make_float2(px, py) : make_float2(0.f, 0.f);
      p.depth[g] = vis ? z : 0.f;
      p.conic[g * 3 + 0] = vis ? __fmul_rn(cc, idet) : 0.f;
      p.conic[g * 3 + 1] = vis ? -__fmul_rn(cb, idet) : 0.f;
      p.conic[g * 3 + 2] = vis ? __fmul_rn(ca, idet) : 0.f;
      p.radius[g] = vis ? static_cast<int>(rad) : 0;
    }
    // view direction and basis values
    float vx = mx - p.cam[0], vy = my - p.cam[1], vz = mz - p.cam[2];
    {
      const float n2 = vx * vx + vy * vy + vz * vz;
      const float in = n2 > 0.f ? rsqrtf(n2) : 0.f;
      vx *= in;
      vy *= in;
      vz *= in;
    }
    float Y[15];
    sh_basis(p.shc, vx, vy, vz, Y);

    const unsigned vm = __ballot_sync(FULL, vis);
    const int nvis = __popc(vm);
    const int rank = __popc(vm & ((1u << lane) - 1u));
    if (vis) vlist[rank] = lane;

    float o0 = 0.f, o1 = 0.f, o2 = 0.f;
    if (CM == CM_SH) {
      __syncwarp();
      if (nvis == GB && p.sh_aligned) {
        // all 32 visible: the batch's rows are one contiguous, 16-byte aligned
        // block of 5760 bytes
        const float4* src = reinterpret_cast<const float4*>(p.sh + base * ROW);
        for (int f = lane; f < GB * ROW / 4; f += 32) cp_async16(stage + 4 * f, src + f);
      } else {
        // copy the visible rows; word f of the stage is word col of row `row`
        int row = 0, col = lane;
        for (int f = lane; f < nvis * ROW; f += 32) {
          cp_async4(stage + f, p.sh + (base + vlist[row]) * ROW + col);
          col += 32;
          if (col >= ROW) {
            col -= ROW;
            ++row;
          }
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncwarp();
      if (vis) {
        const float* yr = stage + rank * ROW;
#pragma unroll
        for (int b = 0; b < 15; ++b) {
          o0 = fmaf(Y[b], yr[b], o0);
          o1 = fmaf(Y[b], yr[15 + b], o1);
          o2 = fmaf(Y[b], yr[30 + b], o2);
        }
      }
    } else {
#pragma unroll
      for (int b = 0; b < 15; ++b) Ys[lane * YS + b] = Y[b];
      Ys[lane * YS + 15] = 0.f;
      nz = nz > s ? s : nz;
      nzs[lane] = nz;
      __syncwarp();  // the batch's codes are staged
      // entries t >= nnz count as zero: clear them, so that the loop below
      // needs no per-entry test
      for (int t = nz; t < s; ++t) cpk[lane * sp + t] = make_uint2(0u, 0u);
      __syncwarp();
      // ---- phase B: 8 lanes per visible Gaussian.  Lane ql owns two bases:
      // FP16 dictionary: 2ql and 2ql+1 (one 16-byte read per nonzero);
      // FP32 dictionary: ql and ql+8 (two 16-byte reads).  In both cases the
      // 8 lanes of a Gaussian read one contiguous 128-byte span per
      // instruction: no bank conflicts.  Basis 15 is the zero slot.
      const int bA = CM == CM_F32 ? ql : 2 * ql, bB = CM == CM_F32 ? ql + 8 : 2 * ql + 1;
      for (int v0 = 0; v0 < nvis; v0 += 4) {
        const int v = v0 + grp;
        const bool act = v < nvis;
        const int gl = act ? vlist[v] : 0;
        const int nzl = act ? nzs[gl] : 0;
        int nzp = max(nzl, __shfl_xor_sync(FULL, nzl, 8));
        nzp = max(nzp, __shfl_xor_sync(FULL, nzp, 16));
        float aR = 0.f, aG = 0.f, aB = 0.f, bR = 0.f, bG = 0.f, bBl = 0.f;
#pragma unroll 2
        for (int t = 0; t < nzp; t += 2) {
          const uint4 c2 = *reinterpret_cast<const uint4*>(cpk + gl * sp + t);
          const uint32_t j0 = c2.x, j1 = c2.z;
          const float a0 = __uint_as_float(c2.y), a1 = __uint_as_float(c2.w);
          if (CM == CM_F32) {
            const float4* D4 = reinterpret_cast<const float4*>(sm);
            const float4 x0 = D4[j0 * 16 + bA], y0 = D4[j0 * 16 + bB];
            const float4 x1 = D4[j1 * 16 + bA], y1 = D4[j1 * 16 + bB];
            aR = fmaf(a0, x0.x, aR);
            aG = fmaf(a0, x0.y, aG);
            aB = fmaf(a0, x0.z, aB);
            bR = fmaf(a0, y0.x, bR);
            bG = fmaf(a0, y0.y, bG);
            bBl = fmaf(a0, y0.z, bBl);
            aR = fmaf(a1, x1.x, aR);
            aG = fmaf(a1, x1.y, aG);
            aB = fmaf(a1, x1.z, aB);
            bR = fmaf(a1, y1.x, bR);
            bG = fmaf(a1, y1.y, bG);
            bBl = fmaf(a1, y1.z, bBl);
          } else {
            // (R, G) and (B, 0) of basis 2ql, then of basis 2ql + 1
            const uint4* D4 = reinterpret_cast<const uint4*>(sm);
            const uint4 w0 = D4[j0 * 8 + ql], w1 = D4[j1 * 8 + ql];
            const float2 rg0 = __half22float2(*reinterpret_cast<const __half2*>(&w0.x));
            const float2 bz0 = __half22float2(*reinterpret_cast<const __half2*>(&w0.y));
            const float2 rh0 = __half22float2(*reinterpret_cast<const __half2*>(&w0.z));
            const float2 bh0 = __half22float2(*reinterpret_cast<const __half2*>(&w0.w));
            const float2 rg1 = __half22float2(*reinterpret_cast<const __half2*>(&w1.x));
            const float2 bz1 = __half22float2(*reinterpret_cast<const __half2*>(&w1.y));
            const float2 rh1 = __half22float2(*reinterpret_cast<const __half2*>(&w1.z));
            const float2 bh1 = __half22float2(*reinterpret_cast<const __half2*>(&w1.w));
            aR = fmaf(a0, rg0.x, aR);
            aG = fmaf(a0, rg0.y, aG);
            aB = fmaf(a0, bz0.x, aB);
            bR = fmaf(a0, rh0.x, bR);
            bG = fmaf(a0, rh0.y, bG);
            bBl = fmaf(a0, bh0.x, bBl);
            aR = fmaf(a1, rg1.x, aR);
            aG = fmaf(a1, rg1.y, aG);
            aB = fmaf(a1, bz1.x, aB);
            bR = fmaf(a1, rh1.x, bR);
            bG = fmaf(a1, rh1.y, bG);
            bBl = fmaf(a1, bh1.x, bBl);
          }
        }
        const float yA = Ys[gl * YS + bA], yB = Ys[gl * YS + bB];
        const float p0 = fmaf(yA, aR, yB * bR), p1 = fmaf(yA, aG, yB * bG), p2 = fmaf(yA, aB, yB * bBl);
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
      if (vis) {
        o0 = outs[lane * 3 + 0];
        o1 = outs[lane * 3 + 1];
        o2 = outs[lane * 3 + 2];
      }
    }
    if (valid) {
      float* out = p.rgb + g * 3;
      out[0] = vis ? fmaxf(0.f, fmaf(p.y00, dr, o0) + 0.5f) : 0.f;
      out[1] = vis ? fmaxf(0.f, fmaf(p.y00, dg, o1) + 0.5f) : 0.f;
      out[2] = vis ? fmaxf(0.f, fmaf(p.y00, db, o2) + 0.5f) : 0.f;
    }
    __syncwarp();
  }
}

static bool aligned(const void* ptr, size_t a) { return (reinterpret_cast<uintptr_t>(ptr) % a) == 0; }

static int fill_common(const dlsh_camera* cam, const dlsh_gaussians* gs, const dlsh_splat_out* out,
                       Params& p, const char* call) {
  if (!cam || !gs || !out) return set_error(DLSH_ERR_INVALID_ARG, "%s: NULL camera, Gaussians or outputs", call);
  if (gs->N < 0) return set_error(DLSH_ERR_INVALID_ARG, "%s: N < 0", call);
  if (gs->N >= (int64_t(1) << 40)) return set_error(DLSH_ERR_UNSUPPORTED, "%s: N too large", call);
  if (!(cam->fx > 0.f) || !(cam->fy > 0.f) || cam->width < 1 || cam->height < 1)
    return set_error(DLSH_ERR_INVALID_ARG, "%s: focal lengths and image size must be positive", call);
  if (gs->N > 0) {
    if (!gs->means || !gs->scales || !gs->quats || !gs->dc || !out->xy || !out->depth || !out->conic ||
        !out->radius || !out->rgb)
      return set_error(DLSH_ERR_INVALID_ARG, "%s: NULL array", call);
    if (!aligned(gs->quats, 16) || !aligned(out->xy, 8))
      return set_error(DLSH_ERR_INVALID_ARG, "%s: quats must be 16-byte and xy 8-byte aligned", call);
  }
  p = Params{};
  p.means = gs->means;
  p.scales = gs->scales;
  p.quats = reinterpret_cast<const float4*>(gs->quats);
  p.dc = gs->dc;
  p.xy = reinterpret_cast<float2*>(out->xy);
  p.depth = out->depth;
  p.conic = out->conic;
  p.radius = out->radius;
  p.rgb = out->rgb;
  p.N = gs->N;
  for (int i = 0; i < 9; ++i) p.R[i] = cam->R[i];
  for (int i = 0; i < 3; ++i) p.t[i] = cam->t[i];
  for (int i = 0; i < 3; ++i)
    p.cam[i] = -(static_cast<double>(cam->R[i]) * cam->t[0] + static_cast<double>(cam->R[3 + i]) * cam->t[1] +
                 static_cast<double>(cam->R[6 + i]) * cam->t[2]);
  p.fx = cam->fx;
  p.fy = cam->fy;
  p.W = static_cast<float>(cam->width);
  p.H = static_cast<float>(cam->height);
  p.hw = 0.5f * p.W;
  p.hh = 0.5f * p.H;
  p.limx = static_cast<float>(kClamp * 0.5 * cam->width / cam->fx);
  p.limy = static_cast<float>(kClamp * 0.5 * cam->height / cam->fy);
  p.z_near = cam->z_near;
  p.y00 = static_cast<float>(0.5 / sqrt(M_PI));
  const ShConst k = make_sh_constants();
  for (int i = 0; i < 15; ++i) p.shc[i] = k.c[i];
  return DLSH_OK;
}

template <int CM>
static int launch(const Params& p, cudaStream_t st, const char* call) {
  if (p.N == 0) return DLSH_OK;
  int sms = device_sm_count();
  if (sms <= 0) sms = 1;
  size_t dbytes = 0, wbytes = 0;
  if (CM == CM_SH) {
    wbytes = static_cast<size_t>(dense_warp_floats()) * 4;
  } else {
    dbytes = static_cast<size_t>(dict_floats(CM, p.K)) * 4;
    wbytes = static_cast<size_t>(codes_warp_floats(p.sp)) * 4;
  }
  int nwarps = static_cast<int>((SMEM_LIMIT - static_cast<long long>(dbytes)) / static_cast<long long>(wbytes));
  if (nwarps > 32) nwarps = 32;
  if (nwarps < 1)
    return set_error(DLSH_ERR_UNSUPPORTED, "%s: K=%d leaves no shared memory for a warp", call, p.K);
  const size_t smem = dbytes + static_cast<size_t>(nwarps) * wbytes;
  DLSH_CUDA_TRY(cudaFuncSetAttribute(preprocess_kernel<CM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SMEM_LIMIT),
                "preprocess: attribute");
  int per_sm = 0;
  DLSH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, preprocess_kernel<CM>, nwarps * 32, smem),
                "preprocess: occupancy");
  if (per_sm < 1) per_sm = 1;
  const int64_t nbatch = (p.N + GB - 1) / GB;
  int64_t grid = static_cast<int64_t>(sms) * per_sm;
  const int64_t need = (nbatch + nwarps - 1) / nwarps;
  if (grid > need) grid = need;
  preprocess_kernel<CM><<<static_cast<int>(grid), nwarps * 32, smem, st>>>(p);
  count_launches(1);
  return check_launch(call);
}

static int check_codes(int K, int s, int64_t N, const float* D, const void* idx, const void* coef,
                       const uint8_t* nnz, const char* call) {
  if (K < 1 || K > DLSH_MAX_K) return set_error(DLSH_ERR_UNSUPPORTED, "%s: K must be in [1, 65535], got %d", call, K);
  if (s < 1 || s > DLSH_MAX_S) return set_error(DLSH_ERR_UNSUPPORTED, "%s: s must be in [1, 32], got %d", call, s);
  if (!D) return set_error(DLSH_ERR_INVALID_ARG, "%s: D is NULL", call);
  if (N > 0 && (!idx || !coef || !nnz)) return set_error(DLSH_ERR_INVALID_ARG, "%s: NULL code array", call);
  return DLSH_OK;
}

static void set_codes(Params& p, const float* D, int K, const void* idx, const void* coef, const uint8_t* nnz,
                      int s) {
  p.D = D;
  p.K = K;
  p.idx = idx;
  p.coef = coef;
  p.nnz = nnz;
  p.s = s;
  p.sp = staged_slots(s);
  p.sdiv = s >= 2 ? static_cast<uint32_t>((uint64_t(1) << 32) / static_cast<uint64_t>(s) + 1) : 0u;
}

}  // namespace spl

size_t preprocess_max_k(int s, int compact) {
  using namespace spl;
  if (s < 1 || s > DLSH_MAX_S) return 0;
  const size_t wb = static_cast<size_t>(codes_warp_floats(staged_slots(s))) * 4;
  const size_t room = static_cast<size_t>(SMEM_LIMIT) - 4 * wb;
  return room / (compact ? 128 : 256);
}

}  // namespace dlsh

extern "C" size_t dlsh_preprocess_max_k(int s, int compact) { return dlsh::preprocess_max_k(s, compact); }

extern "C" int dlsh_preprocess_sh(const dlsh_camera* cam, const dlsh_gaussians* gs, const float* sh,
                                  const dlsh_splat_out* out, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  spl::Params p;
  int rc = spl::fill_common(cam, gs, out, p, "dlsh_preprocess_sh");
  if (rc) return rc;
  if (gs->N > 0 && !sh) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_preprocess_sh: sh is NULL");
  p.sh = sh;
  p.sh_aligned = (reinterpret_cast<uintptr_t>(sh) % 16) == 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = spl::launch<spl::CM_SH>(p, st, "dlsh_preprocess_sh");
  if (rc) return rc;
  return finish(st, nullptr, flags, "dlsh_preprocess_sh");
}

extern "C" int dlsh_preprocess_codes(const dlsh_camera* cam, const dlsh_gaussians* gs, const float* D, int K,
                                     const uint16_t* idx, const float* coef, const uint8_t* nnz, int s,
                                     const dlsh_splat_out* out, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  spl::Params p;
  int rc = spl::fill_common(cam, gs, out, p, "dlsh_preprocess_codes");
  if (rc) return rc;
  rc = spl::check_codes(K, s, gs->N, D, idx, coef, nnz, "dlsh_preprocess_codes");
  if (rc) return rc;
  if (static_cast<size_t>(K) > preprocess_max_k(s, 0))
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_preprocess_codes: K=%d exceeds the shared-memory dictionary (%zu)",
                     K, preprocess_max_k(s, 0));
  spl::set_codes(p, D, K, idx, coef, nnz, s);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = spl::launch<spl::CM_F32>(p, st, "dlsh_preprocess_codes");
  if (rc) return rc;
  return finish(st, nullptr, flags, "dlsh_preprocess_codes");
}

extern "C" int dlsh_preprocess_compact(const dlsh_camera* cam, const dlsh_gaussians* gs, const float* D, int K,
                                       const void* idx, int idx_bytes, const uint16_t* coef_f16,
                                       const uint8_t* nnz, int s, const dlsh_splat_out* out, void* stream,
                                       int flags) {
  using namespace dlsh;
  clear_error();
  spl::Params p;
  int rc = spl::fill_common(cam, gs, out, p, "dlsh_preprocess_compact");
  if (rc) return rc;
  rc = spl::check_codes(K, s, gs->N, D, idx, coef_f16, nnz, "dlsh_preprocess_compact");
  if (rc) return rc;
  if (idx_bytes != 1 && idx_bytes != 2)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_preprocess_compact: idx_bytes must be 1 or 2");
  if (idx_bytes == 1 && K > 256)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_preprocess_compact: 8-bit indices need K <= 256");
  if (static_cast<size_t>(K) > preprocess_max_k(s, 1))
    return set_error(DLSH_ERR_UNSUPPORTED,
                     "dlsh_preprocess_compact: K=%d exceeds the shared-memory dictionary (%zu)", K,
                     preprocess_max_k(s, 1));
  spl::set_codes(p, D, K, idx, coef_f16, nnz, s);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = idx_bytes == 1 ? spl::launch<spl::CM_C8>(p, st, "dlsh_preprocess_compact")
                      : spl::launch<spl::CM_C16>(p, st, "dlsh_preprocess_compact");
  if (rc) return rc;
  return finish(st, nullptr, flags, "dlsh_preprocess_compact");
}
