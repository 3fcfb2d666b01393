// Fused inference of the support-proposal network: for every signal, the m
// atoms with the largest logits of the 45 -> 256 -> 256 -> K GELU MLP, ordered
// by decreasing logit (ties to the smaller atom index), or the logits
// themselves, in one persistent kernel.  Activations never leave the SM.
//
// Per tile of 128 signals (one TMEM lane per signal):
//   epilogue warps  stage the unit-norm BF16 signals as the A operand
//   MMA warp        layer 1 (N = 256, K = 64) into a 256-column TMEM buffer
//   epilogue warps  bias + GELU -> BF16 hidden activations, written over the
//                   A operand in the canonical K-major layout
//   MMA warp        layer 2 (K = 256) into the other TMEM buffer; same epilogue
//   MMA warp        layer 3, 256 atoms per job, TMEM buffers alternating so the
//                   epilogue of one block overlaps the MMAs of the next; in
//                   top-m mode layer 3 runs twice (the tensor pipe has room)
//   epilogue warps  each thread owns one signal and half of every 256-atom
//                   block (8 warps over the 4 TMEM lane quadrants)
//   producer warp   streams the weights, pre-packed into 32 KB operand chunks
//                   in their consumption order, through a 3-stage ring
// The MMAs have the shape of the layer-by-layer training GEMM (M = 128,
// N = 128, K = 16, FP32 accumulation in the same k order) and the element-wise
// steps share its code, so the logits agree with it bit for bit.
//
// Top-m (exact, ties to the smaller atom index):
//   pass A  the maxima of 32 interleaved column groups per half row; the m-th
//           largest of the row's 64 group maxima is a lower bound T of its
//           m-th largest logit (64 distinct logits reach their group maxima)
//   pass B  only logits >= T are queued (shared memory, 16 columns at a time)
//           and inserted into a sorted register list: about m + m^2/128 per
//           row, instead of the m (1 + ln(K/m)) record values of a one-pass scan
//   merge   the two half lists of each signal, by (logit desc, index asc)
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "host.hpp"
#include "internal.hpp"
#include "mlp.cuh"

namespace dlsh {
namespace prop {

using mlp::HID;
using mlp::XIN;

constexpr int TM = 128;                          // signals per tile (MMA M)
constexpr int NC = 256;                          // columns per accumulation job
constexpr int KC = 64;                           // k per operand chunk (four k-steps of 16)
constexpr uint32_t CHUNK_BYTES = NC * KC * 2;    // 32 KB
constexpr int NST = 3;                           // operand ring stages
constexpr int NEPI = 256;                        // epilogue threads (8 warps)
constexpr int NTHREADS = NEPI + 64;              // + MMA warp + producer warp
constexpr int QC = 16;                           // queued logits per thread and flush
constexpr uint32_t A_BYTES = TM * HID * 2;       // 64 KB: X, then H1, then H2
constexpr uint32_t OFF_A = 0;
constexpr uint32_t OFF_RING = OFF_A + A_BYTES;
constexpr uint32_t OFF_Q = OFF_RING + NST * CHUNK_BYTES;
constexpr uint32_t OFF_T = OFF_Q + QC * NEPI * 8;  // per-signal thresholds
constexpr uint32_t OFF_BAR = OFF_T + TM * 4;
constexpr uint32_t SMEM_BYTES = OFF_BAR + 128;
static_assert(SMEM_BYTES <= 232448, "shared memory");
static_assert(QC * NEPI * 8 >= 64 * TM * 4, "the queues hold the sorted group maxima");

// Packed weights: chunk 0 = W1, chunks 1..4 = W2 by k-range, then for each
// 256-atom block j the four k-ranges of W3 rows [256 j, 256 j + 256) (rows
// past K are zero).  Chunk layout: canonical K-major, no swizzle: element
// (n, k) at byte (k / 8) * (NC * 16) + n * 16 + (k % 8) * 2.
inline int n_blocks(int K) { return (K + NC - 1) / NC; }
inline int n_chunks(int K) { return 5 + 4 * n_blocks(K); }

struct Ws {
  uint32_t* status;
  uint8_t* img;
  float* b1;
  float* b2;
  float* b3;  // padded to whole blocks with -inf
};
inline size_t carve(void* base, int K, Ws& w) {
  Carver c(base);
  w.status = c.take<uint32_t>(64);
  w.img = c.take<uint8_t>(static_cast<size_t>(n_chunks(K)) * CHUNK_BYTES);
  w.b1 = c.take<float>(HID);
  w.b2 = c.take<float>(HID);
  w.b3 = c.take<float>(static_cast<size_t>(n_blocks(K)) * NC);
  return c.size();
}

// One thread per 16-byte unit of the image (8 consecutive k of one row).
__global__ void pack_kernel(const __nv_bfloat16* __restrict__ Pb, const float* __restrict__ P, int K,
                            int nblk, uint8_t* __restrict__ img, float* __restrict__ b1,
                            float* __restrict__ b2, float* __restrict__ b3) {
  const mlp::Layout L = mlp::layout(K);
  const long long u = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long units = static_cast<long long>(5 + 4 * nblk) * (CHUNK_BYTES / 16);
  if (u < units) {
    const int c = static_cast<int>(u / (CHUNK_BYTES / 16));
    const int w = static_cast<int>(u % (CHUNK_BYTES / 16));
    const int kb = w / NC, n = w % NC;
    const __nv_bfloat16* src;
    long long row;
    int ld, k0;
    bool valid = true;
    if (c == 0) {
      src = Pb + L.W1;
      ld = XIN;
      row = n;
      k0 = 0;
    } else if (c < 5) {
      src = Pb + L.W2;
      ld = HID;
      row = n;
      k0 = (c - 1) * KC;
    } else {
      const int j = (c - 5) / 4, kc = (c - 5) % 4;
      src = Pb + L.W3;
      ld = HID;
      row = static_cast<long long>(j) * NC + n;
      k0 = kc * KC;
      valid = row < K;
    }
    uint4 v = make_uint4(0, 0, 0, 0);
    if (valid) v = *reinterpret_cast<const uint4*>(src + row * ld + k0 + kb * 8);
    *reinterpret_cast<uint4*>(img + static_cast<size_t>(c) * CHUNK_BYTES + kb * (NC * 16) + n * 16) = v;
  }
  if (u < HID) {
    b1[u] = P[L.b1 + u];
    b2[u] = P[L.b2 + u];
  }
  if (u < static_cast<long long>(nblk) * NC) b3[u] = u < K ? P[L.b3 + u] : -INFINITY;
}

struct Args {
  const float* X;
  long long N;
  const uint8_t* img;
  const float* b1;
  const float* b2;
  const float* b3;
  int nblk, K;
  uint16_t* cand;   // top-m mode: N x m
  float* logits;    // logits mode: N x K, row-major
  uint32_t* status;
  long long budget;
};

// Inserts (z, j) into the sorted list (decreasing logit; equal logits by
// increasing atom index).  z arrives after every listed atom of this thread, so
// it goes below the equal logits: it lands below every entry >= z, and the
// entries under that position shift down one slot, keeping their order.  Only
// z is compared, always against the old entries.  A NaN never enters.
template <int M>
__device__ __forceinline__ void list_insert(float (&tv)[M], int (&tj)[M], float z, int j) {
#pragma unroll
  for (int q = M - 1; q > 0; --q) {
    const bool above = z > tv[q - 1];  // z lands in slot q - 1 or higher
    const bool here = z > tv[q];
    tv[q] = above ? tv[q - 1] : (here ? z : tv[q]);
    tj[q] = above ? tj[q - 1] : (here ? j : tj[q]);
  }
  const bool top = z > tv[0];
  tv[0] = top ? z : tv[0];
  tj[0] = top ? j : tj[0];
}

__device__ __forceinline__ bool ranks_before(float a, int ja, float b, int jb) {
  return a > b || (a == b && ja < jb);
}

// LOGITS = false: the top-M atoms per signal into a.cand.  LOGITS = true: the
// logits themselves into a.logits (the inference forward), same arithmetic.
template <int M, bool LOGITS>
__global__ void __launch_bounds__(NTHREADS, 1) propose_kernel(const __grid_constant__ Args a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* A = smem + OFF_A;
  uint8_t* ring = smem + OFF_RING;
  float2* Q = reinterpret_cast<float2*>(smem + OFF_Q);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OFF_BAR);
  uint64_t* full = bars;              // [NST] chunk landed
  uint64_t* empty = bars + NST;       // [NST] chunk consumed by the MMAs
  uint64_t* tfull = bars + 2 * NST;   // [2] accumulation job done
  uint64_t* tempty = tfull + 2;       // [2] TMEM buffer drained
  uint64_t* abar = tempty + 2;        // A operand written
  uint64_t* mdone = abar + 1;         // every MMA of the issuer complete (exit)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mdone + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long ntiles = (a.N + TM - 1) / TM;
  // layer-3 passes: one in logits mode; two in top-m mode (group maxima for a
  // threshold, then the filtered selection), the MMAs recomputed for the second
  const int passes = LOGITS ? 1 : 2;
  const int jobs = 2 + passes * a.nblk;
  const int nch_tile = 5 + 4 * passes * a.nblk;
  const int nch_img = 5 + 4 * a.nblk;

  if (tid == 0) {
    for (int q = 0; q < NST; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], NEPI / 32);
    }
    mbar_init(abar, NEPI / 32);
    mbar_init(mdone, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == NEPI / 32 + 1) {
    // ------------------------------------------------------ producer
    if (lane == 0) {
      long long ri = 0;
      bool ok = true;
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int c = 0; c < nch_tile; ++c, ++ri) {
          const int ci = c < nch_img ? c : c - 4 * a.nblk;  // the second pass re-reads W3
          const int st = static_cast<int>(ri % NST);
          if (!mbar_wait(&empty[st], static_cast<uint32_t>((ri / NST) & 1) ^ 1u, a.budget)) {
            flag_status(a.status, ST_TIMEOUT);
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[st], CHUNK_BYTES);
          bulk_g2s(ring + st * CHUNK_BYTES, a.img + static_cast<size_t>(ci) * CHUNK_BYTES, CHUNK_BYTES,
                   &full[st]);
        }
      }
      // every issued copy has landed before the CTA may exit
      for (long long f = ri > NST ? ri - NST : 0; f < ri; ++f)
        if (!mbar_wait(&full[f % NST], static_cast<uint32_t>((f / NST) & 1), a.budget))
          flag_status(a.status, ST_TIMEOUT);
    }
  } else if (warp == NEPI / 32) {
    // ------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // N = 128 per instruction, two per k-step: the shape of the training GEMM
      constexpr uint32_t idesc = umma_idesc(1, 1, TM, NC / 2);
      const uint32_t a_addr = smem_u32(A);
      const uint32_t r_addr = smem_u32(ring);
      long long ri = 0, job = 0;
      uint32_t aph = 0;
      bool ok = true, issued = false;
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int L = 0; L < jobs && ok; ++L, ++job) {
          if (L <= 2) {  // layer 1, layer 2, first block of layer 3: a new A operand
            if (!mbar_wait(abar, aph, a.budget)) {
              flag_status(a.status, ST_TIMEOUT);
              ok = false;
              break;
            }
            aph ^= 1u;
          }
          const int b = static_cast<int>(job & 1);
          if (!mbar_wait(&tempty[b], static_cast<uint32_t>((job >> 1) & 1) ^ 1u, a.budget)) {
            flag_status(a.status, ST_TIMEOUT);
            ok = false;
            break;
          }
          tc_fence_after();
          const int nk = L == 0 ? 1 : HID / KC;
          for (int kc = 0; kc < nk; ++kc, ++ri) {
            const int st = static_cast<int>(ri % NST);
            if (!mbar_wait(&full[st], static_cast<uint32_t>((ri / NST) & 1), a.budget)) {
              flag_status(a.status, ST_TIMEOUT);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t bb = r_addr + static_cast<uint32_t>(st) * CHUNK_BYTES;
#pragma unroll
            for (int ks = 0; ks < KC / 16; ++ks) {
              const uint64_t ad = umma_smem_desc(a_addr + (kc * 8 + ks * 2) * (TM * 16), TM * 16, 128);
#pragma unroll
              for (int nh = 0; nh < 2; ++nh) {
                const uint64_t bd =
                    umma_smem_desc(bb + ks * 2 * (NC * 16) + nh * (NC / 2) * 16, NC * 16, 128);
                umma_bf16(tmem + static_cast<uint32_t>(b * NC + nh * (NC / 2)), ad, bd, idesc,
                          (kc | ks) ? 1u : 0u);
              }
            }
            issued = true;
            tc_commit(&empty[st]);
          }
          if (ok) tc_commit(&tfull[b]);
        }
      }
      if (issued) {  // no MMA may still write TMEM when it is released
        tc_commit(mdone);
        if (!mbar_wait(mdone, 0, a.budget)) flag_status(a.status, ST_TIMEOUT);
      }
    }
  } else {
    // ------------------------------------------------------ epilogue warps
    const int q4 = warp & 3;             // TMEM lane quadrant
    const int h = warp >> 2;             // column half of each 256-column job
    const int r = q4 * 32 + lane;        // the thread's signal within the tile
    const uint32_t tl = tmem + (static_cast<uint32_t>(q4 * 32) << 16);
    float2* LST = reinterpret_cast<float2*>(A);  // merge lists, [half * M + e][128]
    long long job = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      // ---- signals -> unit-norm BF16 rows of A (k < 64); warp w: rows 16w..16w+15
      {
        float x0[16], x1[16];
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) {
          const long long g = tile * TM + warp * 16 + rr;
          x0[rr] = g < a.N ? a.X[g * DLSH_D + lane] : 0.f;
          x1[rr] = (g < a.N && lane < DLSH_D - 32) ? a.X[g * DLSH_D + 32 + lane] : 0.f;
        }
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) {
          __nv_bfloat16 y0, y1;
          mlp::normalise_pair(x0[rr], x1[rr], y0, y1);
          const int row = warp * 16 + rr;
          *reinterpret_cast<__nv_bfloat16*>(A + (lane >> 3) * (TM * 16) + row * 16 + (lane & 7) * 2) = y0;
          *reinterpret_cast<__nv_bfloat16*>(A + ((32 + lane) >> 3) * (TM * 16) + row * 16 + (lane & 7) * 2) = y1;
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(abar);
      }
      // ---- layers 1 and 2: bias + GELU, BF16 activations over A
      for (int layer = 0; layer < 2; ++layer, ++job) {
        const int b = static_cast<int>(job & 1);
        if (ok && !mbar_wait(&tfull[b], static_cast<uint32_t>((job >> 1) & 1), a.budget)) {
          flag_status(a.status, ST_TIMEOUT);
          ok = false;
        }
        tc_fence_after();
        const float* bias = layer == 0 ? a.b1 : a.b2;
        if (ok) {
#pragma unroll 1
          for (int p = 0; p < 4; ++p) {
            const int c0 = h * 128 + p * 32;
            float v[32];
            tmem_ld32(tl + static_cast<uint32_t>(b * NC + c0), v);
            const float4* bp = reinterpret_cast<const float4*>(bias + c0);
#pragma unroll
            for (int g8 = 0; g8 < 4; ++g8) {
              const float4 bA = __ldg(bp + 2 * g8), bB = __ldg(bp + 2 * g8 + 1);
              const float bb[8] = {bA.x, bA.y, bA.z, bA.w, bB.x, bB.y, bB.z, bB.w};
              uint32_t pk[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const __nv_bfloat16 lo =
                    __float2bfloat16(mlp::gelu_f(mlp::add_bias(v[g8 * 8 + 2 * e], bb[2 * e])));
                const __nv_bfloat16 hi =
                    __float2bfloat16(mlp::gelu_f(mlp::add_bias(v[g8 * 8 + 2 * e + 1], bb[2 * e + 1])));
                pk[e] = static_cast<uint32_t>(__bfloat16_as_ushort(lo)) |
                        (static_cast<uint32_t>(__bfloat16_as_ushort(hi)) << 16);
              }
              *reinterpret_cast<uint4*>(A + ((c0 >> 3) + g8) * (TM * 16) + r * 16) =
                  make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
          }
        }
        tc_fence_before();
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&tempty[b]);
          mbar_arrive(abar);
        }
      }
      // ---- layer 3
      float tv[M];
      int tj[M];
#pragma unroll
      for (int q = 0; q < M; ++q) {
        tv[q] = -INFINITY;
        tj[q] = 0x7fffffff;
      }
      float T = -INFINITY;
      if constexpr (!LOGITS) {
        // pass A: maxima of 32 interleaved groups (column mod 32) of the thread's
        // half row
        float gmax[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) gmax[i] = -INFINITY;
        for (int j = 0; j < a.nblk; ++j, ++job) {
          const int b = static_cast<int>(job & 1);
          if (ok && !mbar_wait(&tfull[b], static_cast<uint32_t>((job >> 1) & 1), a.budget)) {
            flag_status(a.status, ST_TIMEOUT);
            ok = false;
          }
          tc_fence_after();
          if (ok) {
            const uint32_t tb = tl + static_cast<uint32_t>(b * NC + h * 128);
            const float* bias = a.b3 + static_cast<size_t>(j) * NC + h * 128;
#pragma unroll 1
            for (int p = 0; p < 4; ++p) {
              float v[32];
              tmem_ld32(tb + p * 32, v);
              const float4* bp = reinterpret_cast<const float4*>(bias + p * 32);
#pragma unroll
              for (int i4 = 0; i4 < 8; ++i4) {
                const float4 bq = __ldg(bp + i4);
                const float bb[4] = {bq.x, bq.y, bq.z, bq.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                  gmax[i4 * 4 + e] = fmaxf(gmax[i4 * 4 + e], mlp::add_bias(v[i4 * 4 + e], bb[e]));
              }
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[b]);
        }
        // sort the 32 maxima (bitonic network, decreasing), publish them, and
        // let the h = 0 thread merge both halves' lists up to the M-th element
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
          for (int jj = k >> 1; jj > 0; jj >>= 1) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const int l = i ^ jj;
              if (l > i) {
                const float x = gmax[i], y = gmax[l];
                const bool dec = (i & k) == 0;
                gmax[i] = dec ? fmaxf(x, y) : fminf(x, y);
                gmax[l] = dec ? fminf(x, y) : fmaxf(x, y);
              }
            }
          }
        }
        float* S = reinterpret_cast<float*>(Q);  // [half * 32 + rank][128]
        float* Ts = reinterpret_cast<float*>(smem + OFF_T);
#pragma unroll
        for (int i = 0; i < 32; ++i) S[(h * 32 + i) * TM + r] = gmax[i];
        named_bar_sync(1, NEPI);
        if (h == 0) {
          int i0 = 0, i1 = 0;
          float t = -INFINITY;
#pragma unroll 1
          for (int q = 0; q < M; ++q) {
            const float x = S[i0 * TM + r], y = S[(32 + i1) * TM + r];
            const bool take1 = y > x;
            t = take1 ? y : x;
            i1 += take1 ? 1 : 0;
            i0 += take1 ? 0 : 1;
          }
          Ts[r] = t;
        }
        named_bar_sync(1, NEPI);
        T = Ts[r];
      }
      // pass B (the only pass in logits mode)
      for (int j = 0; j < a.nblk; ++j, ++job) {
        const int b = static_cast<int>(job & 1);
        if (ok && !mbar_wait(&tfull[b], static_cast<uint32_t>((job >> 1) & 1), a.budget)) {
          flag_status(a.status, ST_TIMEOUT);
          ok = false;
        }
        tc_fence_after();
        const uint32_t tb = tl + static_cast<uint32_t>(b * NC + h * 128);
        const float* bias = a.b3 + static_cast<size_t>(j) * NC + h * 128;
        if (ok && LOGITS) {
          const long long g = tile * TM + r;
#pragma unroll 1
          for (int p = 0; p < 4; ++p) {
            float v[32];
            tmem_ld32(tb + p * 32, v);
            const int a0 = j * NC + h * 128 + p * 32;
            if (g < a.N) {
              float* out = a.logits + g * a.K + a0;
#pragma unroll
              for (int i = 0; i < 32; ++i)
                if (a0 + i < a.K) out[i] = mlp::add_bias(v[i], __ldg(bias + p * 32 + i));
            }
          }
        } else if (ok) {
          // queue the logits >= T, 16 columns at a time, then insert them
#pragma unroll 1
          for (int p = 0; p < 4; ++p) {
            float v[32];
            tmem_ld32(tb + p * 32, v);
            const float4* bp = reinterpret_cast<const float4*>(bias + p * 32);
            const int a0 = j * NC + h * 128 + p * 32;
#pragma unroll
            for (int hp = 0; hp < 2; ++hp) {
              int cnt = 0;
#pragma unroll
              for (int i4 = 0; i4 < 4; ++i4) {
                const float4 bq = __ldg(bp + hp * 4 + i4);
                const float bb[4] = {bq.x, bq.y, bq.z, bq.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  const int i = hp * 16 + i4 * 4 + e;
                  const float z = mlp::add_bias(v[i], bb[e]);
                  if (z >= T) {
                    Q[cnt * NEPI + tid] = make_float2(z, __int_as_float(a0 + i));
                    ++cnt;
                  }
                }
              }
              const int mx = __reduce_max_sync(0xffffffffu, cnt);
              for (int e = 0; e < mx; ++e) {
                if (e < cnt) {
                  const float2 qe = Q[e * NEPI + tid];
                  if (qe.x > tv[M - 1]) list_insert<M>(tv, tj, qe.x, __float_as_int(qe.y));
                }
              }
              T = fmaxf(T, tv[M - 1]);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
      }
      // ---- merge the two halves (A is free: every MMA of the tile is done; in
      // logits mode it takes the next signals right away)
      if (named_bar_or(1, NEPI, !ok)) break;
      if constexpr (!LOGITS) {
#pragma unroll
        for (int q = 0; q < M; ++q) LST[(h * M + q) * TM + r] = make_float2(tv[q], __int_as_float(tj[q]));
        named_bar_sync(1, NEPI);
        const long long g = tile * TM + r;
        if (h == 0 && g < a.N) {
          int i0 = 0, i1 = 0;
          uint32_t pk[(M + 1) / 2];
#pragma unroll
          for (int q = 0; q < (M + 1) / 2; ++q) pk[q] = 0u;
#pragma unroll
          for (int q = 0; q < M; ++q) {
            const float2 e0 = LST[(i0 < M ? i0 : M - 1) * TM + r];
            const float2 e1 = LST[(M + (i1 < M ? i1 : M - 1)) * TM + r];
            const int j0 = __float_as_int(e0.y), j1 = __float_as_int(e1.y);
            const bool take1 = i0 >= M || (i1 < M && ranks_before(e1.x, j1, e0.x, j0));
            const int jj = take1 ? j1 : j0;
            i1 += take1 ? 1 : 0;
            i0 += take1 ? 0 : 1;
            pk[q >> 1] |= static_cast<uint32_t>(static_cast<uint16_t>(jj)) << (16 * (q & 1));
          }
          uint16_t* out = a.cand + g * M;
          if constexpr (M >= 8) {
#pragma unroll
            for (int q = 0; q < M / 8; ++q)
              reinterpret_cast<uint4*>(out)[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
          } else if constexpr (M == 4) {
            *reinterpret_cast<uint2*>(out) = make_uint2(pk[0], pk[1]);
          } else {
            *reinterpret_cast<uint32_t*>(out) = pk[0];
          }
        }
        named_bar_sync(1, NEPI);  // the lists are read before A takes the next signals
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace prop

size_t propose_ws_bytes(int K) {
  prop::Ws w;
  return prop::carve(nullptr, K, w);
}

// Packs the weights, then launches the fused kernel: top-m into cand (m > 0)
// or the logits into `logits` (m = 0).
static int fused_enqueue(const void* mlp_blob, int K, const float* X, long long N, int m,
                         uint16_t* cand, float* logits, void* ws, uint32_t* status, cudaStream_t st,
                         const char* call) {
  using namespace prop;
  if (reinterpret_cast<uintptr_t>(ws) % 256)
    return set_error(DLSH_ERR_INVALID_ARG, "%s: workspace must be 256-byte aligned", call);
  mlp::Blob b;
  mlp::carve_blob(const_cast<void*>(mlp_blob), K, b);
  Ws w;
  carve(ws, K, w);
  const int nblk = n_blocks(K);
  const long long units = static_cast<long long>(n_chunks(K)) * (CHUNK_BYTES / 16);
  pack_kernel<<<static_cast<int>((units + 255) / 256), 256, 0, st>>>(b.Pb, b.P, K, nblk, w.img, w.b1,
                                                                     w.b2, w.b3);
  count_launches(1);
  int rc = check_launch(call);
  if (rc) return rc;
  Args a;
  a.X = X;
  a.N = N;
  a.img = w.img;
  a.b1 = w.b1;
  a.b2 = w.b2;
  a.b3 = w.b3;
  a.nblk = nblk;
  a.K = K;
  a.cand = cand;
  a.logits = logits;
  a.status = status;
  a.budget = kWaitBudget;
  const long long ntiles = (N + TM - 1) / TM;
  const int grid = static_cast<int>(ntiles < device_sm_count() ? ntiles : device_sm_count());
#define LAUNCH(MM, LG)                                                                             \
  do {                                                                                             \
    static PerDevice<int> attr;                                                                    \
    int attr_ok = 0;                                                                               \
    const int arc = attr.get(&attr_ok, [&](int& v) {                                               \
      DLSH_CUDA_TRY(cudaFuncSetAttribute(propose_kernel<MM, LG>,                                   \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES), \
                    call);                                                                         \
      v = 1;                                                                                       \
      return DLSH_OK;                                                                              \
    });                                                                                            \
    if (arc) return arc;                                                                           \
    propose_kernel<MM, LG><<<grid, NTHREADS, SMEM_BYTES, st>>>(a);                                 \
  } while (0)
  switch (m) {
    case 0: LAUNCH(2, true); break;
    case 2: LAUNCH(2, false); break;
    case 4: LAUNCH(4, false); break;
    case 8: LAUNCH(8, false); break;
    case 16: LAUNCH(16, false); break;
    default: LAUNCH(32, false); break;
  }
#undef LAUNCH
  count_launches(1);
  return check_launch(call);
}

int propose_enqueue(const void* mlp_blob, int K, const float* X, long long N, int m, uint16_t* cand,
                    void* ws, uint32_t* status, cudaStream_t st) {
  if (m != 2 && m != 4 && m != 8 && m != 16 && m != 32)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_mlp_propose: m must be 2, 4, 8, 16 or 32");
  if (N <= 0) return DLSH_OK;
  if (reinterpret_cast<uintptr_t>(cand) % (2 * m < 16 ? 2 * m : 16))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_mlp_propose: cand must be aligned to min(16, 2m) bytes");
  return fused_enqueue(mlp_blob, K, X, N, m, cand, nullptr, ws, status, st, "dlsh_mlp_propose");
}

int infer_logits_enqueue(const void* mlp_blob, int K, const float* X, long long N, float* logits,
                         void* ws, uint32_t* status, cudaStream_t st) {
  if (N <= 0) return DLSH_OK;
  return fused_enqueue(mlp_blob, K, X, N, 0, nullptr, logits, ws, status, st, "dlsh_mlp_forward");
}

}  // namespace dlsh
