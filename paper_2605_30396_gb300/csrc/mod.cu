// Dictionary update with the codes fixed (Sec. 2.1: alternating minimisation of
// Eq. 1), read as MOD: the least-squares minimiser of sum ||x_i - D alpha_i||^2
// in D, with a small ridge so that unused atoms keep it well posed:
//   G = A A^T, B = X A^T, lambda = 1e-6 trace(G)/K,
//   D~^T = (G + lambda I)^-1 (B + lambda D_old)^T, d_j = d~_j / ||d~_j||,
//   unused atoms refilled with the worst-fit signals.
//
// GPU design (deterministic, no floating-point atomics):
//   1. count_kernel     per-tile atom histograms (integer counts)
//   2. scan kernels     per-atom totals, atom offsets, per-(atom, tile) offsets
//   3. scatter_kernel   one CTA per signal tile writes (signal, coef, nnz) into
//                       the atom-major list in signal order (a counting sort)
//   4. accum_kernel     one CTA per segment of an atom's list: row j of G
//                       (entries k >= j; G is symmetric, and its lower
//                       triangle is mirrored from the upper one after the
//                       reduction) and column j of B.  Each warp owns a fixed slice, one list
//                       entry per lane pair; sums are float-float (exact FMA
//                       products, two-sum accumulation: about FP64 accuracy
//                       on the FP32 pipe, since GB300's FP64 units are slow),
//                       lanes and warps are added in a fixed order
//   5. mixed-precision solve of (G + lambda I) D~^T = (B + lambda D_old)^T:
//      Jacobi scaling S = diag^-1/2 (unit diagonal); one cooperative kernel
//      factors S (G + lambda I) S = L L^T in FP32 and inverts L on the way
//      (right-looking steps over [A | I], a grid barrier between phases);
//      each FP32 solve is then two triangular products with W = L^-1, and
//      iterative refinement uses the residual of the scaled system computed
//      in FP64 (GB300's FP64 rate is a small fraction of its FP32 rate, so
//      FP64 is spent only there)
//   6. normalise, then refill unused atoms (argmax passes over resid_sq)
//
// The same file holds the other reading of the D-step, the approximate K-SVD
// sweep (dlsh_ksvd_update): it reuses the counting sort (1-3, with each
// record's code slot), then runs the atoms in order on one cooperative kernel,
// and refills unused atoms as in 6.
#include <math.h>

#include "common.cuh"
#include "host.hpp"
#include "internal.hpp"

namespace dlsh {
namespace mod {

constexpr int TS = 512;        // signals per counting-sort tile (one scatter CTA each)
constexpr int NB = 32;         // Cholesky block
constexpr int RW = 48;         // padded RHS width (45 used)
constexpr int MAX_K = 4096;    // shared-memory G-row partials limit
constexpr int SMEM_LIMIT = 232448;
constexpr double RIDGE_REL = 1e-6;
constexpr int kRefine = 3;     // FP32 solves (two FP64 residual corrections)

struct Ws {
  uint32_t* status;
  int* cnt;        // K x T per-(atom, tile) counts
  int* off;        // K x T offsets
  int* atom_total; // K
  int* atom_start; // K + 1
  uint2* list;     // N*s atom-major records: (signal | nnz << 26, coefficient bits)
  double* M;       // K x K: G + lambda I (FP64, kept for the refinement residuals)
  double* Z;       // K x RW: B^T (lambda D_old is added where Z is read)
  double* lam;     // [0] lambda
  double* dsc;     // K: Jacobi scale 1 / sqrt(M_jj)
  float* A32;      // K x K: S M S, then its FP32 Cholesky factor (lower)
  float* W32;      // K x K: L^-1 (lower)
  float* Y32;      // K x RW: W r, between the two triangular products
  unsigned* gbar;  // grid barrier of the factorisation: arrivals, generation
  double* Zs;      // K x RW: S Z
  double* Xs;      // K x RW: solution of the scaled system (FP64 accumulation)
  float* R32;      // K x RW: current residual of the scaled system
  double* Xb;      // K x RW: D~^T = S Xs, kept up to date with Xs
  int* dead;       // K
  int* seg_start;  // P*K + 1: first accumulation segment of each (block p, atom j), p-major
  double* Gp;      // max_segs x K partial G rows
  double* Bp;      // max_segs x RW partial B columns
};

constexpr int SEG = 4096;  // list entries per accumulation segment
// Signals per accumulation block: segments never cross a block, and the grid
// walks the blocks in order.  Blocks of 262,144 signals (47 MB of rows, held
// in L2 while gathered) measured slower on GB300 than whole-list segments:
// the gathers are not the binding limit, the per-segment work is.  The value
// here puts every atom's list in one block.
constexpr int64_t BLK = int64_t(1) << 40;
static_assert(BLK % TS == 0, "blocks are whole counting-sort tiles");

inline int64_t n_blocks(int64_t N) { return N > 0 ? (N + BLK - 1) / BLK : 1; }
// counting-sort tiles per block, capped at the tile count (fits an int)
inline int tiles_per_block(int64_t T) { return static_cast<int>(BLK / TS < T ? BLK / TS : T); }
inline int64_t max_segments(int K, int s, int64_t N) {
  return (N * s + SEG - 1) / SEG + n_blocks(N) * K;
}

static size_t carve(void* base, int K, int s, int64_t N, Ws& w) {
  Carver c(base);
  const int64_t T = (N + TS - 1) / TS > 0 ? (N + TS - 1) / TS : 1;
  w.status = c.take<uint32_t>(64);
  w.cnt = c.take<int>(static_cast<size_t>(K) * T);
  w.off = c.take<int>(static_cast<size_t>(K) * T);
  w.atom_total = c.take<int>(K);
  w.atom_start = c.take<int>(K + 1);
  w.list = c.take<uint2>(static_cast<size_t>(N) * s + 1);
  w.M = c.take<double>(static_cast<size_t>(K) * K);
  w.Z = c.take<double>(static_cast<size_t>(K) * RW);
  w.lam = c.take<double>(4);
  w.dsc = c.take<double>(K);
  w.A32 = c.take<float>(static_cast<size_t>(K) * K);
  w.W32 = c.take<float>(static_cast<size_t>(K) * K);
  w.Y32 = c.take<float>(static_cast<size_t>(K) * RW);
  w.gbar = c.take<unsigned>(64);
  w.Zs = c.take<double>(static_cast<size_t>(K) * RW);
  w.Xs = c.take<double>(static_cast<size_t>(K) * RW);
  w.R32 = c.take<float>(static_cast<size_t>(K) * RW);
  w.Xb = c.take<double>(static_cast<size_t>(K) * RW);
  w.dead = c.take<int>(K);
  w.seg_start = c.take<int>(static_cast<size_t>(n_blocks(N)) * K + 1);
  w.Gp = c.take<double>(static_cast<size_t>(max_segments(K, s, N)) * K);
  w.Bp = c.take<double>(static_cast<size_t>(max_segments(K, s, N)) * RW);
  return c.size();
}

// ---- float-float accumulation: (hi, lo) += a * b, product exact via FMA ------
__device__ __forceinline__ void ff_fma(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float v = __fadd_rn(s, -hi);
  float e = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -v)), __fadd_rn(p, -v));
  e = __fadd_rn(e, __fadd_rn(lo, pe));
  hi = __fadd_rn(s, e);
  lo = __fadd_rn(e, -__fadd_rn(hi, -s));
}

// ---- 1. per-tile histograms ------------------------------------------------
__global__ void count_kernel(const uint16_t* __restrict__ idx, const uint8_t* __restrict__ nnz,
                             int s, int64_t N, int K, int T, int* __restrict__ cnt,
                             uint32_t* status) {
  extern __shared__ int hist[];
  for (int j = threadIdx.x; j < K; j += blockDim.x) hist[j] = 0;
  __syncthreads();
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * TS;
  const int nt = static_cast<int>(N - i0 < TS ? N - i0 : TS);  // signals in this tile
  const uint16_t* tidx = idx + i0 * s;
  bool bad = false;
#pragma unroll 4
  for (int e = threadIdx.x; e < nt * s; e += blockDim.x) {
    const int q = e / s;
    const int t = e - q * s;
    int nz = nnz[i0 + q];
    if (nz > s) {
      bad = true;
      nz = s;
    }
    if (t < nz) {
      const int j = tidx[e];
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

// ---- 2. offsets: per-atom totals, atom starts, per-(atom, tile) offsets -------
__device__ __forceinline__ int block_exclusive_scan(int v, int* sm, int* total) {
  // Hillis-Steele over blockDim.x (<= 1024) values; returns the exclusive prefix
  const int tid = threadIdx.x;
  sm[tid] = v;
  __syncthreads();
  for (int o = 1; o < static_cast<int>(blockDim.x); o <<= 1) {
    const int u = tid >= o ? sm[tid - o] : 0;
    __syncthreads();
    sm[tid] += u;
    __syncthreads();
  }
  const int incl = sm[tid];
  if (total) *total = sm[blockDim.x - 1];
  __syncthreads();
  return incl - v;
}

__global__ void atom_total_kernel(const int* __restrict__ cnt, int T, int* __restrict__ atom_total) {
  __shared__ int red[256];
  const int j = blockIdx.x;
  int acc = 0;
  for (int b = threadIdx.x; b < T; b += blockDim.x) acc += cnt[static_cast<size_t>(j) * T + b];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (static_cast<int>(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atom_total[j] = red[0];
}

__global__ void atom_scan_kernel(const int* __restrict__ atom_total, int K,
                                 int* __restrict__ atom_start) {
  __shared__ int sm[1024];
  __shared__ int carry_s;
  int carry = 0;
  for (int base = 0; base < K; base += 1024) {
    const int j = base + threadIdx.x;
    const int v = j < K ? atom_total[j] : 0;
    int tot = 0;
    const int ex = block_exclusive_scan(v, sm, &tot);
    if (j < K) atom_start[j] = carry + ex;
    if (threadIdx.x == 0) carry_s = carry + tot;
    __syncthreads();
    carry = carry_s;
    __syncthreads();
  }
  if (threadIdx.x == 0) atom_start[K] = carry;
}

__global__ void tile_offsets_kernel(const int* __restrict__ cnt, int T,
                                    const int* __restrict__ atom_start, int* __restrict__ off) {
  __shared__ int sm[256];
  const int j = blockIdx.x;
  const int per = (T + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per, b1 = b0 + per < T ? b0 + per : T;
  int sum = 0;
  for (int b = b0; b < b1; ++b) sum += cnt[static_cast<size_t>(j) * T + b];
  int run = atom_start[j] + block_exclusive_scan(sum, sm, nullptr);
  for (int b = b0; b < b1; ++b) {
    off[static_cast<size_t>(j) * T + b] = run;
    run += cnt[static_cast<size_t>(j) * T + b];
  }
}

// ---- 3. counting-sort scatter, one CTA of 8 warps per tile, signal order ------
// The tile's code indices and counts are first staged in shared memory with
// coalesced loads, so that neither pass waits on a chain of dependent global
// loads.  Warp w owns signals [64 w, 64 w + 64) of the tile and walks their code
// slots in order, 32 at a time.  Pass 1 counts each atom per warp (lanes with
// the same atom found by match-any); the counts become per-warp bases; pass 2
// gives each entry its rank among the earlier entries of its atom (warps in
// order, then lanes in order) and writes it to the atom-major list.  A signal's
// atoms are distinct, so within an atom the entries stay in signal order.
// SLOT: the record's upper 6 bits hold the entry's code slot t instead of nnz.
constexpr int SC_T = 256;
// Shared memory of a scatter CTA: staged indices (TS s uint16, a multiple of 16
// bytes), counts (TS bytes), then per-warp counts [8][K] and tile offsets [K].
inline size_t scatter_smem(int K, int s) {
  return static_cast<size_t>(TS) * s * 2 + TS + static_cast<size_t>(SC_T / 32 + 1) * K * sizeof(int);
}
template <bool SLOT>
__global__ void __launch_bounds__(SC_T) scatter_kernel(const uint16_t* __restrict__ idx,
                                                      const float* __restrict__ coef,
                                                      const uint8_t* __restrict__ nnz, int s, int64_t N,
                                                      int K, int T, const int* __restrict__ off,
                                                      uint2* __restrict__ list) {
  extern __shared__ __align__(16) uint8_t scb[];
  uint16_t* sidx = reinterpret_cast<uint16_t*>(scb);                        // [TS * s]
  uint8_t* snz = scb + static_cast<size_t>(TS) * s * 2;                     // [TS]
  int* wc = reinterpret_cast<int*>(snz + TS);                               // [8][K] counts, then bases
  int* toff = wc + static_cast<size_t>(SC_T / 32) * K;                      // [K] this tile's list offsets
  const int b = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t t0 = static_cast<int64_t>(b) * TS;
  const int nt = static_cast<int>(N - t0 < TS ? N - t0 : TS);  // signals in this tile
  {
    // 16-byte loads where the tile's index rows are 16-byte aligned (the tile
    // starts at a multiple of TS s, so only the array's base decides), the rest
    // element by element
    const uint16_t* src = idx + t0 * s;
    const int ne = nt * s;
    int done = 0;
    if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
      const int nv = ne / 8;
      for (int v = tid; v < nv; v += SC_T)
        reinterpret_cast<uint4*>(sidx)[v] = __ldg(reinterpret_cast<const uint4*>(src) + v);
      done = nv * 8;
    }
    for (int e = done + tid; e < ne; e += SC_T) sidx[e] = src[e];
    for (int q = tid; q < nt; q += SC_T) snz[q] = nnz[t0 + q];
  }
  for (int j = tid; j < K; j += SC_T) {
    toff[j] = off[static_cast<size_t>(j) * T + b];
#pragma unroll
    for (int w = 0; w < SC_T / 32; ++w) wc[w * K + j] = 0;
  }
  __syncthreads();
  constexpr int SPW = TS / (SC_T / 32);  // signals per warp (64)
  const int q0 = warp * SPW;              // the warp's first signal in the tile
  const int64_t i0 = t0 + q0;
  const int qn = nt - q0 < SPW ? nt - q0 : SPW;
  const int e_end = (qn > 0 ? qn : 0) * s;  // <= 64 * 32
  int* mine = wc + static_cast<size_t>(warp) * K;
  const unsigned lt = (1u << lane) - 1u;
  // entry e of the warp: its atom j (-1 if none), coefficient c (only when
  // with_coef), count or slot field nz and signal
  auto entry = [&](int e, bool with_coef, int& j, float& c, int& nz, int64_t& sig) {
    j = -1;
    c = 0.f;
    nz = 0;
    sig = 0;
    if (e < e_end) {
      const int q = e / s;
      sig = i0 + q;
      const int t = e - q * s;
      nz = snz[q0 + q];
      nz = nz > s ? s : nz;
      const bool live = t < nz;
      if (SLOT) nz = t;
      if (live) {
        const int jj = sidx[(q0 + q) * s + t];
        if (jj < K) {
          j = jj;
          if (with_coef) c = coef[sig * s + t];
        }
      }
    }
  };
  // pass 1: counts
  for (int e0 = 0; e0 < e_end; e0 += 32) {
    int j, nz;
    float c;
    int64_t sig;
    entry(e0 + lane, false, j, c, nz, sig);
    const unsigned m = __match_any_sync(0xffffffffu, j);
    if (j >= 0 && (m & lt) == 0) mine[j] += __popc(m);
    __syncwarp();
  }
  __syncthreads();
  // per-warp bases: warps in order
  for (int j = tid; j < K; j += SC_T) {
    int run = toff[j];
#pragma unroll
    for (int w = 0; w < SC_T / 32; ++w) {
      const int cw = wc[w * K + j];
      wc[w * K + j] = run;
      run += cw;
    }
  }
  __syncthreads();
  // pass 2: ranks and writes
  for (int e0 = 0; e0 < e_end; e0 += 32) {
    int j, nz;
    float c;
    int64_t sig;
    entry(e0 + lane, true, j, c, nz, sig);
    const unsigned m = __match_any_sync(0xffffffffu, j);
    if (j >= 0) {
      const int pos = mine[j] + __popc(m & lt);
      list[pos] = make_uint2(static_cast<uint32_t>(sig) | (static_cast<uint32_t>(nz) << 26), __float_as_uint(c));
    }
    __syncwarp();
    if (j >= 0 && (m & lt) == 0) mine[j] += __popc(m);
    __syncwarp();
  }
}

// ---- 4. G row j and B column j ---------------------------------------------------
// Entry range [lo, hi) of atom j's list that lies in signal block p (tpb
// counting-sort tiles per block).
__device__ __forceinline__ void block_range(const int* __restrict__ off,
                                            const int* __restrict__ atom_start, int T, int tpb,
                                            int j, int p, int& lo, int& hi) {
  const int t0 = p * tpb, t1 = t0 + tpb;
  lo = t0 < T ? off[static_cast<size_t>(j) * T + t0] : atom_start[j + 1];
  hi = t1 < T ? off[static_cast<size_t>(j) * T + t1] : atom_start[j + 1];
}

// One CTA per accumulation segment (a slice of atom j's list inside one signal
// block); the warps split the segment, one list entry per lane pair and 16
// entries per step:
//   B   each lane keeps float-float sums of its entries' a_ij x_i over half of
//       the 45 dimensions in registers (the signal row is read straight from
//       global memory); a butterfly of two-sums adds the lanes up at the end
//   G   for each support slot t with atom k > j, the lanes add a_ij a_ik into
//       the warp's row partial in shared memory (the entries k < j come from
//       row k's segments, mirrored later); lanes that hit the same atom k are
//       grouped (match) and their products summed in lane order by the group's
//       first lane before its single update; the diagonal k = j stays in
//       registers
// Every sum runs in a fixed order, so the result does not depend on timing.
__device__ __forceinline__ void ff_add(float& h, float& l, float p, float pl) {
  const float s = __fadd_rn(h, p);
  const float v = __fadd_rn(s, -h);
  const float e = __fadd_rn(__fadd_rn(h, -__fadd_rn(s, -v)), __fadd_rn(p, -v));
  const float t = __fadd_rn(e, __fadd_rn(l, pl));
  h = __fadd_rn(s, t);
  l = __fadd_rn(t, -__fadd_rn(h, -s));
}

// SMAX >= s: the support slots of a lane's entry are loaded into registers at
// the start of each step, next to its signal row, so no load waits inside the
// slot loop.  Two lanes share an entry (half of its dimensions and slots each),
// which halves the registers and doubles the warps an SM can hold: five CTAs
// per SM at s <= 8 (96 registers a thread), four at s <= 16.
constexpr int DH = (DLSH_D + 1) / 2;  // dimensions per lane of a pair (23)
template <int SMAX>
__global__ void __launch_bounds__(128, SMAX <= 8 ? 5 : (SMAX <= 16 ? 4 : 3))
    accum_kernel(const float* __restrict__ X, const uint16_t* __restrict__ idx,
                 const float* __restrict__ coef, int s, int K, const int* __restrict__ atom_start,
                 const int* __restrict__ off, int T, int tpb, int PK,
                 const int* __restrict__ seg_start, const uint2* __restrict__ list,
                 double* __restrict__ Gp, double* __restrict__ Bp) {
  extern __shared__ __align__(16) float smf[];
  const int nw = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  float* ghi = smf + static_cast<size_t>(warp) * 2 * K;
  float* glo = ghi + K;
  double* bpart = reinterpret_cast<double*>(smf + static_cast<size_t>(nw) * 2 * K) + warp * RW;
  const int nseg = seg_start[PK];
  for (int seg = blockIdx.x; seg < nseg; seg += gridDim.x) {
    // the segment's (block, atom): the largest pj with seg_start[pj] <= seg
    int pj = 0;
    {
      int lo = 0, hi = PK - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_start[mid] <= seg) lo = mid; else hi = mid - 1;
      }
      pj = lo;
    }
    const int pb = pj / K, j = pj - pb * K;
    for (int k = lane; k < K; k += 32) {
      ghi[k] = 0.f;
      glo[k] = 0.f;
    }
    __syncwarp();
    int rlo, rhi;
    block_range(off, atom_start, T, tpb, j, pb, rlo, rhi);
    const int e0 = rlo + (seg - seg_start[pj]) * SEG;
    const int e1 = e0 + SEG < rhi ? e0 + SEG : rhi;
    const int len = e1 - e0;
    const int q0 = e0 + static_cast<int>(static_cast<long long>(len) * warp / nw);
    const int q1 = e0 + static_cast<int>(static_cast<long long>(len) * (warp + 1) / nw);
    // lane pair (2p, 2p + 1) takes entry p of each step of 16: the even lane
    // dimensions 0..22 and slots 0..SMAX/2-1, the odd lane the rest
    const int sub = lane & 1, pe = lane >> 1;
    const int d0 = sub * DH;
    float bh[DH], bl[DH];
#pragma unroll
    for (int d = 0; d < DH; ++d) {
      bh[d] = 0.f;
      bl[d] = 0.f;
    }
    float dh = 0.f, dl = 0.f;  // G[j][j]
    constexpr int SH = SMAX / 2;
    // the next step's list record is loaded one step ahead, and its signal row
    // and code slots are prefetched into L2 while this step computes
    uint2 rec_next = make_uint2(0u, 0u);
    if (q0 + pe < q1) rec_next = list[q0 + pe];
    for (int eb = q0; eb < q1; eb += 16) {
      const int e = eb + pe;
      const bool act = e < q1;
      const uint2 rec = rec_next;
      if (eb + 16 + pe < q1) {
        rec_next = list[eb + 16 + pe];
        const long long sn = static_cast<long long>(rec_next.x & 0x3FFFFFFu);
        const char* xr = reinterpret_cast<const char*>(X + sn * DLSH_D);
        if (sub == 0) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(xr));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(xr + 92));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(xr + 176));
        } else {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(idx + sn * s));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(coef + sn * s));
        }
      }
      long long sig = 0;
      int nz = 0;
      float a = 0.f;
      if (act) {
        sig = static_cast<long long>(rec.x & 0x3FFFFFFu);
        nz = static_cast<int>(rec.x >> 26);
        a = __uint_as_float(rec.y);
      }
      int kk[SH];
      float cc[SH];
      {
        const uint16_t* ir = idx + sig * s;
        const float* cr = coef + sig * s;
#pragma unroll
        for (int u = 0; u < SH; ++u) {
          const int t = sub * SH + u;
          const bool on = act && t < nz;
          kk[u] = on ? static_cast<int>(__ldg(ir + t)) : -1;
          cc[u] = on ? __ldg(cr + t) : 0.f;
        }
      }
      if (act) {
        const float* xr = X + sig * DLSH_D + d0;
        float xv[DH];
#pragma unroll
        for (int d = 0; d < DH; ++d) xv[d] = (d0 + d < DLSH_D) ? __ldg(xr + d) : 0.f;
#pragma unroll
        for (int d = 0; d < DH; ++d) ff_fma(bh[d], bl[d], a, xv[d]);
      }
      const int mine = act ? (nz - sub * SH < 0 ? 0 : (nz - sub * SH > SH ? SH : nz - sub * SH)) : 0;
      const int mx = __reduce_max_sync(FULL, mine);
#pragma unroll
      for (int u = 0; u < SH; ++u) {
        if (u >= mx) break;  // uniform over the warp
        const bool on = kk[u] >= 0;
        const int k = kk[u];
        const float c = cc[u];
        if (on && k == j) ff_fma(dh, dl, a, c);
        const bool upd = on && k > j && k < K;
        const unsigned m = __ballot_sync(FULL, upd);
        if (upd) {
          const unsigned grp = __match_any_sync(m, k);
          float ph = __fmul_rn(a, c);
          float pl = __fmaf_rn(a, c, -ph);
          const int first = __ffs(grp) - 1;
          if (grp != (1u << lane)) {
            // the group's products, summed in lane order on its first lane
            unsigned rest = grp & ~(1u << first);
            float sh = ph, sl = pl;
            while (rest) {
              const int src = __ffs(rest) - 1;
              const float h2 = __shfl_sync(grp, ph, src);
              const float l2 = __shfl_sync(grp, pl, src);
              ff_add(sh, sl, h2, l2);
              rest &= rest - 1;
            }
            ph = sh;
            pl = sl;
          }
          if (lane == first) {
            float h = ghi[k], l = glo[k];
            ff_add(h, l, ph, pl);
            ghi[k] = h;
            glo[k] = l;
          }
        }
        __syncwarp();
      }
    }
    // the lanes' sums: butterflies of two-sums, B over the lanes of equal
    // parity (their dimensions agree), the diagonal over all lanes
#pragma unroll
    for (int d = 0; d < DH; ++d)
#pragma unroll
      for (int o = 16; o > 1; o >>= 1) {
        const float h2 = __shfl_xor_sync(FULL, bh[d], o);
        const float l2 = __shfl_xor_sync(FULL, bl[d], o);
        ff_add(bh[d], bl[d], h2, l2);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(FULL, dh, o);
      const float l2 = __shfl_xor_sync(FULL, dl, o);
      ff_add(dh, dl, h2, l2);
    }
    if (lane == 0) {
      float h = ghi[j], l = glo[j];
      ff_add(h, l, dh, dl);
      ghi[j] = h;
      glo[j] = l;
    }
    {
      // lanes 0 and 1 store the two halves.  Every index here is a constant:
      // a lane-dependent pick of bh[d] would make the compiler keep bh and bl
      // in local memory for the whole kernel.
      if (pe == 0) {
#pragma unroll
        for (int d = 0; d < DH; ++d)
          if (d0 + d < DLSH_D) bpart[d0 + d] = static_cast<double>(bh[d]) + static_cast<double>(bl[d]);
      }
      if (lane < RW - DLSH_D) bpart[DLSH_D + lane] = 0.0;
    }
    // sum the warps' partials in order, in float-float (FP64 arithmetic is
    // slow on this part: one conversion pair and one add per atom instead of
    // four)
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      float h = smf[k], l = smf[K + k];
      for (int w = 1; w < nw; ++w) {
        const float* gh = smf + static_cast<size_t>(w) * 2 * K;
        ff_add(h, l, gh[k], gh[K + k]);
      }
      Gp[static_cast<size_t>(seg) * K + k] = static_cast<double>(h) + static_cast<double>(l);
    }
    for (int q = threadIdx.x; q < RW; q += blockDim.x) {
      double acc = 0.0;
      for (int w = 0; w < nw; ++w)
        acc += reinterpret_cast<const double*>(smf + static_cast<size_t>(nw) * 2 * K)[w * RW + q];
      Bp[static_cast<size_t>(seg) * RW + q] = acc;
    }
    __syncthreads();  // shared partials are reused by the next segment
  }
}

// M's lower triangle from its upper one: row j of G holds the entries k >= j,
// so M[k][j] = M[j][k] for k > j (32 x 32 tiles through shared memory; only
// the tiles on or above the diagonal are read).
constexpr int MT = 32;
__global__ void __launch_bounds__(MT * 8) mirror_kernel(double* __restrict__ M, int K) {
  __shared__ double t[MT][MT + 1];
  const int rb = blockIdx.y, cb = blockIdx.x;  // source tile: rows rb, columns cb >= rb
  if (cb < rb) return;
  const int x = threadIdx.x % MT, y0 = threadIdx.x / MT;
  for (int y = y0; y < MT; y += 8) {
    const int r = rb * MT + y, c = cb * MT + x;
    t[y][x] = (r < K && c < K) ? M[static_cast<size_t>(r) * K + c] : 0.0;
  }
  __syncthreads();
  // destination: row cb*MT + y, column rb*MT + x, written where it lies below
  // the diagonal
  for (int y = y0; y < MT; y += 8) {
    const int r = cb * MT + y, c = rb * MT + x;
    if (r < K && c < K && r > c) M[static_cast<size_t>(r) * K + c] = t[x][y];
  }
}

// Segment counts per (block p, atom j) (ceil(n_pj / SEG)) and their exclusive
// scan, p-major.
__global__ void seg_scan_kernel(const int* __restrict__ off, const int* __restrict__ atom_start,
                                int T, int tpb, int K, int PK, int* __restrict__ seg_start) {
  __shared__ int sm[1024];
  __shared__ int carry_s;
  int carry = 0;
  for (int base = 0; base < PK; base += 1024) {
    const int pj = base + threadIdx.x;
    int v = 0;
    if (pj < PK) {
      const int p = pj / K, j = pj - p * K;
      int lo, hi;
      block_range(off, atom_start, T, tpb, j, p, lo, hi);
      v = (hi - lo + SEG - 1) / SEG;
    }
    int tot = 0;
    const int ex = block_exclusive_scan(v, sm, &tot);
    if (pj < PK) seg_start[pj] = carry + ex;
    if (threadIdx.x == 0) carry_s = carry + tot;
    __syncthreads();
    carry = carry_s;
    __syncthreads();
  }
  if (threadIdx.x == 0) seg_start[PK] = carry;
}

// Row j of G and column j of B: the atom's segment partials summed in order.
__global__ void seg_reduce_kernel(const int* __restrict__ seg_start, const double* __restrict__ Gp,
                                  const double* __restrict__ Bp, int K, int P,
                                  double* __restrict__ M, double* __restrict__ Z) {
  const int j = blockIdx.x;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double acc = 0.0;
    for (int p = 0; p < P; ++p)
      for (int sg = seg_start[p * K + j]; sg < seg_start[p * K + j + 1]; ++sg)
        acc += Gp[static_cast<size_t>(sg) * K + k];
    M[static_cast<size_t>(j) * K + k] = acc;
  }
  for (int q = threadIdx.x; q < RW; q += blockDim.x) {
    double acc = 0.0;
    for (int p = 0; p < P; ++p)
      for (int sg = seg_start[p * K + j]; sg < seg_start[p * K + j + 1]; ++sg)
        acc += Bp[static_cast<size_t>(sg) * RW + q];
    Z[static_cast<size_t>(j) * RW + q] = acc;
  }
}

static int accum_warps(int K, int s, size_t* smem) {
  (void)s;
  for (int nw = 4; nw >= 1; --nw) {
    const size_t b = static_cast<size_t>(nw) * 2 * K * 4 + static_cast<size_t>(nw) * RW * 8;
    if (b <= static_cast<size_t>(SMEM_LIMIT)) {
      *smem = b;
      return nw;
    }
  }
  return 0;
}

// ---- 5a. lambda = 1e-6 trace(G)/K (applied where M and Z are read) ----------
__global__ void ridge_kernel(const double* __restrict__ M, int K, double* lam_out) {
  __shared__ double part[1024];
  double acc = 0.0;
  for (int j = threadIdx.x; j < K; j += blockDim.x) acc += M[static_cast<size_t>(j) * K + j];
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {  // fixed-order tree (blockDim.x = 1024)
    if (static_cast<int>(threadIdx.x) < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double tr = part[0];
    *lam_out = tr > 0.0 ? RIDGE_REL * tr / K : RIDGE_REL;
  }
}

// ---- 5b. Jacobi scaling: S = diag(M)^-1/2, A = S M S (FP32, lower), Zs = S Z --
// One CTA per row j.  A has a unit diagonal, which keeps the FP32 factorisation
// well scaled; the refinement below works on the same scaled system in FP64.
// M and Z stay as accumulated; lambda enters here and in the residuals:
// (M + lambda I) and (Z + lambda D_old).
__global__ void scale_kernel(const double* __restrict__ M, const double* __restrict__ Z,
                             const float* __restrict__ D_old, const double* __restrict__ lamp, int K,
                             double* __restrict__ dsc, float* __restrict__ A,
                             double* __restrict__ Zs, float* __restrict__ R32,
                             double* __restrict__ Xs, double* __restrict__ Xb) {
  const int j = blockIdx.x;
  const double lam = *lamp;
  const double dj = 1.0 / sqrt(M[static_cast<size_t>(j) * K + j] + lam);
  if (threadIdx.x == 0) dsc[j] = dj;
  for (int k = threadIdx.x; k <= j; k += blockDim.x) {
    const double dk = 1.0 / sqrt(M[static_cast<size_t>(k) * K + k] + lam);
    const double m = M[static_cast<size_t>(j) * K + k] + (k == j ? lam : 0.0);
    A[static_cast<size_t>(j) * K + k] = static_cast<float>(dj * m * dk);
  }
  for (int c = threadIdx.x; c < RW; c += blockDim.x) {
    const double z = c < DLSH_D ? dj * (Z[static_cast<size_t>(j) * RW + c] +
                                        lam * static_cast<double>(D_old[static_cast<size_t>(j) * DLSH_D + c]))
                                : 0.0;
    Zs[static_cast<size_t>(j) * RW + c] = z;
    R32[static_cast<size_t>(j) * RW + c] = static_cast<float>(z);
    Xs[static_cast<size_t>(j) * RW + c] = 0.0;
    Xb[static_cast<size_t>(j) * RW + c] = 0.0;
  }
}

// ---- 5c. FP32 Cholesky of A and the inverse of its factor, W = L^-1 ----------
// One cooperative launch (every CTA resident) walks the 32-column steps of a
// right-looking factorisation of the augmented matrix [A | I]:
//   phase 1  each CTA factors the diagonal block in one warp (L_kk and its
//            inverse); the grid computes the panel L_ik = A_ik L_kk^-T (i > k)
//            and the rows W_k = L_kk^-1 R_k of the inverse
//   phase 2  CTA 0 stores L_kk; trailing update A_ij -= L_ik L_jk^T (j <= i)
//            and right-hand sides R_i -= L_ik W_k (i > k), on 64 x 64 tiles
//            spread over the CTAs
// with a grid barrier after each phase.  After the last step A holds L and W
// holds L^-1 (lower; its upper triangle stays exactly zero), so every later
// solve is two triangular products, parallel over the whole matrix.
constexpr int CH_T = 256;   // threads per CTA
constexpr int CH_TILE = 64;

// One warp factors the nb x nb diagonal block at k0 (rows past K padded with
// the identity): L into Ls, L^-1 into Li (both lower, [32][33]).  Lane r holds
// row r in registers; pivots and entries move by shuffles.  Every loop is
// unrolled over the full block so that the rows stay in registers, and the
// pivots use the hardware reciprocal square root: the FP64 refinement of the
// solve absorbs its last-bit error.
__device__ void factor_diag(const float* __restrict__ A, int K, int k0, int nb, float (*Ls)[NB + 1],
                            float (*Li)[NB + 1], bool& bad) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  float a[NB], il[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k)
    a[k] = (lane < nb && k < nb) ? (k <= lane ? A[static_cast<size_t>(k0 + lane) * K + k0 + k] : 0.f)
                                 : (k == lane ? 1.f : 0.f);
  bad = false;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    float d = __shfl_sync(FULL, a[c], c);
    if (!(d > 0.f)) {
      bad = true;
      d = 1e-30f;
    }
    const float r = rsqrtf(d);
    il[c] = r;  // 1 / L[c][c]
    a[c] = lane == c ? d * r : (lane > c ? a[c] * r : a[c]);  // L[lane][c]
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      if (k > c) {
        const float lkc = __shfl_sync(FULL, a[c], k);  // L[k][c]
        a[k] = lane >= k ? fmaf(-a[c], lkc, a[k]) : a[k];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NB; ++k) Ls[lane][k] = k <= lane ? a[k] : 0.f;
  // X = L^-1, one column per lane: X[r][c] = (delta_rc - sum_{k<r} L[r][k] X[k][c]) / L[r][r]
  float x[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    float acc = r == lane ? 1.f : 0.f;
#pragma unroll
    for (int k = 0; k < NB; ++k)
      if (k < r) acc = fmaf(-__shfl_sync(FULL, a[k], r), x[k], acc);
    x[r] = r >= lane ? acc * il[r] : 0.f;
  }
#pragma unroll
  for (int r = 0; r < NB; ++r) Li[r][lane] = x[r];
}

// C[64 x 64 tile] -= P Q^T over 32 k: P rows from pload(r, q), Q rows from
// qload(c, q), both staged transposed; 4 x 4 outputs per thread, applied by
// cupd(r, c, value).
template <class PF, class QF, class CF>
__device__ __forceinline__ void tile_update(float (*Ps)[CH_TILE + 1], float (*Qs)[CH_TILE + 1], PF pload,
                                            QF qload, CF cupd) {
  for (int f = threadIdx.x; f < CH_TILE * NB; f += CH_T) {
    const int r = f / NB, q = f % NB;
    Ps[q][r] = pload(r, q);
    Qs[q][r] = qload(r, q);
  }
  __syncthreads();
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;  // rows tr + 16i, cols tc + 16j
  float acc[4][4] = {};
#pragma unroll 8
  for (int q = 0; q < NB; ++q) {
    float pi[4], qj[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) pi[i] = Ps[q][tr + 16 * i];
#pragma unroll
    for (int j = 0; j < 4; ++j) qj[j] = Qs[q][tc + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(pi[i], qj[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) cupd(tr + 16 * i, tc + 16 * j, acc[i][j]);
  __syncthreads();  // the staging tiles are reused by the next tile
}

__global__ void __launch_bounds__(CH_T) chol_inv_kernel(float* __restrict__ A, float* __restrict__ W, int K,
                                                        unsigned* __restrict__ bar,
                                                        uint32_t* __restrict__ status, long long budget) {
  __shared__ float Ls[NB][NB + 1];
  __shared__ float Li[NB][NB + 1];
  __shared__ float Ps[NB][CH_TILE + 1];
  __shared__ float Qs[NB][CH_TILE + 1];
  const int tid = threadIdx.x;
  const long long gt = static_cast<long long>(blockIdx.x) * CH_T + tid;
  const long long gstride = static_cast<long long>(gridDim.x) * CH_T;
  // W = I (the augmented right-hand sides)
  for (long long e = gt; e < static_cast<long long>(K) * K; e += gstride)
    W[e] = (e / K == e % K) ? 1.f : 0.f;
  if (!grid_barrier(bar, budget, status)) return;
  const int nblk = (K + NB - 1) / NB;
  for (int kb = 0; kb < nblk; ++kb) {
    const int k0 = kb * NB, nb = K - k0 < NB ? K - k0 : NB, k1 = k0 + nb;
    // ---- phase 1 (the diagonal block is read by every CTA: nobody writes it here)
    if (tid < 32) {
      bool bad = false;
      factor_diag(A, K, k0, nb, Ls, Li, bad);
      if (bad && tid == 0 && blockIdx.x == 0) flag_status(status, ST_BAD_INPUT);
    }
    __syncthreads();
    // Warp tasks over the whole grid: the panel rows (lane c, holding row c of
    // L_kk^-1 in registers: L_ic = sum_q A_iq Li[c][q]) and 32-column tiles of
    // the rows of W (one column per lane: W_qc = sum_p Li[q][p] R_pc).
    {
      const int lane = tid & 31;
      float lr[NB];
#pragma unroll
      for (int q = 0; q < NB; ++q) lr[q] = Li[lane][q];
      const int gw = blockIdx.x * (CH_T / 32) + (tid >> 5);
      const int nwarps = gridDim.x * (CH_T / 32);
      const int npanel = K - k1;
      const int ntiles = (k1 + 31) / 32;
      for (int task = gw; task < npanel + ntiles; task += nwarps) {
        if (task < npanel) {
          const int i = k1 + task;
          float* ar = A + static_cast<size_t>(i) * K + k0;
          const float v = lane < nb ? ar[lane] : 0.f;
          float acc = 0.f;
#pragma unroll
          for (int q = 0; q < NB; ++q) acc = fmaf(__shfl_sync(0xffffffffu, v, q), lr[q], acc);
          if (lane < nb) ar[lane] = acc;
        } else {
          // lane c: column c0 + c of R_k, y_q = sum_{p <= q} Li[q][p] R_pc
          const int c = (task - npanel) * 32 + lane;
          if (c < k1) {
            float r[NB];
#pragma unroll
            for (int p = 0; p < NB; ++p) r[p] = p < nb ? W[static_cast<size_t>(k0 + p) * K + c] : 0.f;
#pragma unroll
            for (int q = 0; q < NB; ++q) {
              if (q < nb) {
                float acc = 0.f;
#pragma unroll
                for (int p = 0; p <= q; ++p) acc = fmaf(Li[q][p], r[p], acc);
                W[static_cast<size_t>(k0 + q) * K + c] = acc;
              }
            }
          }
        }
      }
    }
    if (!grid_barrier(bar, budget, status)) return;
    // ---- phase 2: the factored diagonal block, the trailing update of A
    // (lower tiles) and of the right-hand sides
    if (blockIdx.x == 0 && tid < nb)
      for (int k = 0; k < nb; ++k) A[static_cast<size_t>(k0 + tid) * K + k0 + k] = Ls[tid][k];
    const int rest = K - k1;  // > 0 only when nb = NB (a partial block is the last)
    if (rest > 0) {
      const int T1 = (rest + CH_TILE - 1) / CH_TILE;
      const int T2 = (k1 + CH_TILE - 1) / CH_TILE;
      const int nsyrk = T1 * (T1 + 1) / 2;
      const int total = nsyrk + T1 * T2;
      for (int t = blockIdx.x; t < total; t += gridDim.x) {
        if (t < nsyrk) {
          int bi = static_cast<int>((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
          while (bi * (bi + 1) / 2 > t) --bi;
          while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
          const int bj = t - bi * (bi + 1) / 2;
          const int r0 = k1 + bi * CH_TILE, c0 = k1 + bj * CH_TILE;
          tile_update(
              Ps, Qs,
              [&](int r, int q) { return r0 + r < K ? A[static_cast<size_t>(r0 + r) * K + k0 + q] : 0.f; },
              [&](int r, int q) { return c0 + r < K ? A[static_cast<size_t>(c0 + r) * K + k0 + q] : 0.f; },
              [&](int r, int c, float v) {
                const int gr = r0 + r, gc = c0 + c;
                if (gr < K && gc <= gr) A[static_cast<size_t>(gr) * K + gc] -= v;
              });
        } else {
          const int u = t - nsyrk;
          const int bi = u / T2, bc = u % T2;
          const int r0 = k1 + bi * CH_TILE, c0 = bc * CH_TILE;
          tile_update(
              Ps, Qs,
              [&](int r, int q) { return r0 + r < K ? A[static_cast<size_t>(r0 + r) * K + k0 + q] : 0.f; },
              [&](int c, int q) {
                return (c0 + c < k1 && q < nb) ? W[static_cast<size_t>(k0 + q) * K + c0 + c] : 0.f;
              },
              [&](int r, int c, float v) {
                const int gr = r0 + r, gc = c0 + c;
                if (gr < K && gc < k1) W[static_cast<size_t>(gr) * K + gc] -= v;
              });
        }
      }
    }
    if (!grid_barrier(bar, budget, status)) return;
  }
}

// ---- 5d. FP32 solve of (L L^T) c = r with W = L^-1: y = W r, then c = W^T y,
// and X += c in FP64.  One warp per output row: the lanes split the inner index,
// each keeps the row's 48 partial sums, and a butterfly adds them up.  No
// shared memory and no block barriers: every row proceeds independently.
template <bool TRANS>
__global__ void __launch_bounds__(256) trmm_kernel(const float* __restrict__ W, int K,
                                                   const float* __restrict__ in, float* __restrict__ out,
                                                   double* __restrict__ Xs, const double* __restrict__ dsc,
                                                   double* __restrict__ Xb) {
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= K) return;
  float acc[RW];
#pragma unroll
  for (int c = 0; c < RW; ++c) acc[c] = 0.f;
  // W lower: y_i = sum_{j <= i} W_ij r_j;  W^T: c_j = sum_{i >= j} W_ij y_i
  const int k_begin = TRANS ? row : 0;
  const int k_end = TRANS ? K : row + 1;
  for (int k = k_begin + lane; k < k_end; k += 32) {
    const float w = TRANS ? W[static_cast<size_t>(k) * K + row] : W[static_cast<size_t>(row) * K + k];
    const float4* v = reinterpret_cast<const float4*>(in + static_cast<size_t>(k) * RW);
#pragma unroll
    for (int q = 0; q < RW / 4; ++q) {
      const float4 x = v[q];
      acc[4 * q] = fmaf(w, x.x, acc[4 * q]);
      acc[4 * q + 1] = fmaf(w, x.y, acc[4 * q + 1]);
      acc[4 * q + 2] = fmaf(w, x.z, acc[4 * q + 2]);
      acc[4 * q + 3] = fmaf(w, x.w, acc[4 * q + 3]);
    }
  }
#pragma unroll
  for (int c = 0; c < RW; ++c)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
  // every lane holds every sum; lane l stores columns l and 32 + l
  float v0 = 0.f, v1 = 0.f;
#pragma unroll
  for (int c = 0; c < 32; ++c) v0 = lane == c ? acc[c] : v0;
#pragma unroll
  for (int c = 32; c < RW; ++c) v1 = lane == c - 32 ? acc[c] : v1;
  if (TRANS) {
    // the solution and its unscaled form D~^T = S Xs, which the FP64 residual
    // and the normalisation read
    const size_t o = static_cast<size_t>(row) * RW;
    const double dr = dsc[row];
    const double x0 = Xs[o + lane] + static_cast<double>(v0);
    Xs[o + lane] = x0;
    Xb[o + lane] = dr * x0;
    if (lane < DLSH_D - 32) {
      const double x1 = Xs[o + 32 + lane] + static_cast<double>(v1);
      Xs[o + 32 + lane] = x1;
      Xb[o + 32 + lane] = dr * x1;
    }
  } else {
    out[static_cast<size_t>(row) * RW + lane] = v0;
    if (lane < RW - 32) out[static_cast<size_t>(row) * RW + 32 + lane] = v1;
  }
}

// ---- 5e. FP64 residual of the scaled system: R = Zs - (S M S) X, as FP32 -----
// 8 x 48 output tiles (K/8 CTAs, so the FP64 pipes of every SM take part);
// thread (row tid / 24, columns tid % 24 and tid % 24 + 24); k in chunks of 32.
constexpr int RS_ROWS = 8;
constexpr int RS_T = 256;   // four groups of 64 threads split each k chunk
__global__ void __launch_bounds__(RS_T) residual_kernel(const double* __restrict__ M,
                                                        const double* __restrict__ lamp,
                                                        const double* __restrict__ dsc, int K,
                                                        const double* __restrict__ Zs,
                                                        const double* __restrict__ Xb,
                                                        float* __restrict__ R32) {
  __shared__ double Ms[RS_ROWS][33];
  __shared__ double Xt[32][RW + 1];
  __shared__ double red[4][RS_ROWS][RW];
  const int j0 = blockIdx.x * RS_ROWS;
  const double lam = *lamp;
  const int g = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int r0 = (t >> 4) * 2, c0 = (t & 15) * 3;  // 2 rows x 3 columns per thread
  double acc[2][3] = {};
  for (int k0 = 0; k0 < K; k0 += 32) {
    {
      const int r = threadIdx.x / 32, c = threadIdx.x % 32;
      Ms[r][c] = (j0 + r < K && k0 + c < K)
                     ? M[static_cast<size_t>(j0 + r) * K + k0 + c] + (j0 + r == k0 + c ? lam : 0.0)
                     : 0.0;
    }
    for (int f = threadIdx.x; f < 32 * RW; f += RS_T) {
      const int r = f / RW, c = f % RW;
      Xt[r][c] = k0 + r < K ? Xb[static_cast<size_t>(k0 + r) * RW + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const int k = kk * 4 + g;
      const double m0 = Ms[r0][k], m1 = Ms[r0 + 1][k];
      const double x0 = Xt[k][c0], x1 = Xt[k][c0 + 1], x2 = Xt[k][c0 + 2];
      acc[0][0] = fma(m0, x0, acc[0][0]);
      acc[0][1] = fma(m0, x1, acc[0][1]);
      acc[0][2] = fma(m0, x2, acc[0][2]);
      acc[1][0] = fma(m1, x0, acc[1][0]);
      acc[1][1] = fma(m1, x1, acc[1][1]);
      acc[1][2] = fma(m1, x2, acc[1][2]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) red[g][r0 + i][c0 + jj] = acc[i][jj];
  __syncthreads();
  // the four k groups in a fixed order
  for (int f = threadIdx.x; f < RS_ROWS * RW; f += RS_T) {
    const int r = f / RW, c = f % RW;
    const int j = j0 + r;
    if (j < K) {
      const double sum = ((red[0][r][c] + red[1][r][c]) + red[2][r][c]) + red[3][r][c];
      R32[static_cast<size_t>(j) * RW + c] = static_cast<float>(Zs[static_cast<size_t>(j) * RW + c] - dsc[j] * sum);
    }
  }
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
  __shared__ int dl[MAX_K];   // the dead atoms, increasing
  __shared__ int wcount[32];
  __shared__ float prev_v;
  __shared__ long long prev_i;
  __shared__ int found, ndead;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  if (tid == 0) {
    prev_v = INFINITY;
    prev_i = -1;
    ndead = 0;
  }
  __syncthreads();
  // ordered compaction of the dead flags (one pass of ballots per 1024 atoms)
  for (int base = 0; base < K; base += 1024) {
    const bool d = base + tid < K && dead[base + tid] != 0;
    const unsigned m = __ballot_sync(0xffffffffu, d);
    if (lane == 0) wcount[wp] = __popc(m);
    __syncthreads();
    int before = ndead;
    for (int q = 0; q < wp; ++q) before += wcount[q];
    if (d) dl[before + __popc(m & ((1u << lane) - 1u))] = base + tid;
    __syncthreads();
    if (tid == 0)
      for (int q = 0; q < 32; ++q) ndead += wcount[q];
    __syncthreads();
  }
  for (int t = 0; t < ndead; ++t) {
    const int j = dl[t];
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

// ---- approximate K-SVD (the alternative D-update) ------------------------------
// A sweep over the atoms in order; atom j and the coefficients that use it are
// refitted with one power step from the current coefficients g (Rubinstein,
// Zibulevsky and Elad, 2008):
//   E = R_w + g d_j^T (R = X - D A, kept current),  d = E^T g / ||E^T g||,
//   g' = E d,  R_w <- E - g' d^T,  d_j <- d,  A[j, w] <- g'.
// R lives in the workspace, rows padded to 48 floats (16-byte loads).  One
// cooperative kernel runs the sweep: per atom, every thread takes list entries
// lo + tid, lo + tid + (grid threads), ...; phase 1 sums g R_i and g^2 (per
// thread, then a transposing butterfly per warp, then the warps and the CTAs
// in a fixed order: the result does not depend on timing); a grid barrier;
// phase 2 forms d in every CTA and updates R, the coefficients and the atom; a
// second grid barrier before the next atom reads R.  The atom-major list
// records each entry's code slot, so the coefficient is written directly.
constexpr int KS_T = 256;          // threads per sweep CTA
constexpr int KS_W = KS_T / 32;
constexpr int RROW = 48;           // residual row stride in floats
constexpr int KS_V = DLSH_D + 1;   // reduced values: 45 of g R_i, then g^2

struct KsWs {
  uint32_t* status;
  int* cnt;
  int* off;
  int* atom_total;
  int* atom_start;
  uint2* list;
  float* R;        // N x 48 residual (45 used)
  float* part;     // grid x 48 per-CTA partial sums
  int* dead;
  unsigned* gbar;
};

constexpr int KS_MAX_GRID = 1024;

static size_t carve_ksvd(void* base, int K, int s, int64_t N, KsWs& w) {
  Carver c(base);
  const int64_t T = (N + TS - 1) / TS > 0 ? (N + TS - 1) / TS : 1;
  w.status = c.take<uint32_t>(64);
  w.cnt = c.take<int>(static_cast<size_t>(K) * T);
  w.off = c.take<int>(static_cast<size_t>(K) * T);
  w.atom_total = c.take<int>(K);
  w.atom_start = c.take<int>(K + 1);
  w.list = c.take<uint2>(static_cast<size_t>(N) * s + 1);
  w.R = c.take<float>(static_cast<size_t>(N) * RROW);
  w.part = c.take<float>(static_cast<size_t>(KS_MAX_GRID) * 48);
  w.dead = c.take<int>(K);
  w.gbar = c.take<unsigned>(64);
  return c.size();
}

// R = X - D A with the input codes; one warp per signal, lane d owning
// dimensions d and d + 32 (and the zero padding 45..47).
__global__ void __launch_bounds__(256) ksvd_resid_kernel(const float* __restrict__ X, const float* __restrict__ D,
                                                         int K, const uint16_t* __restrict__ idx,
                                                         const float* __restrict__ coef,
                                                         const uint8_t* __restrict__ nnz, int s, int64_t N,
                                                         float* __restrict__ R) {
  const int lane = threadIdx.x & 31;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= N) return;
  const bool hi = lane < DLSH_D - 32;
  float r0 = X[i * DLSH_D + lane];
  float r1 = hi ? X[i * DLSH_D + 32 + lane] : 0.f;
  int nz = nnz[i];
  nz = nz > s ? s : nz;
  const int jl = lane < nz ? idx[i * s + lane] : 0;
  const float al = lane < nz ? coef[i * s + lane] : 0.f;
  for (int t = 0; t < nz; ++t) {
    const int j = __shfl_sync(0xffffffffu, jl, t);
    const float a = __shfl_sync(0xffffffffu, al, t);
    if (j >= K) continue;
    const float* dr = D + static_cast<size_t>(j) * DLSH_D;
    r0 = fmaf(-a, dr[lane], r0);
    if (hi) r1 = fmaf(-a, dr[32 + lane], r1);
  }
  R[i * RROW + lane] = r0;
  if (lane < RROW - 32) R[i * RROW + 32 + lane] = r1;
}

__global__ void __launch_bounds__(KS_T) ksvd_sweep_kernel(const int* __restrict__ atom_start,
                                                          const uint2* __restrict__ list, int K, int s,
                                                          float* __restrict__ coef, const float* __restrict__ D_old,
                                                          float* __restrict__ D_new, float* __restrict__ R,
                                                          float* __restrict__ part, int* __restrict__ dead,
                                                          unsigned* gbar, uint32_t* status, long long budget) {
  extern __shared__ float pall[];  // [gridDim.x][48] the CTAs' partial sums, phase 2
  __shared__ float wsum[KS_W][64];
  __shared__ __align__(16) float dj[RROW], dn[RROW];
  __shared__ float tot[48];
  __shared__ float dd_s;
  __shared__ int skip_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t gthreads = static_cast<int64_t>(gridDim.x) * KS_T;
  const int64_t gtid = static_cast<int64_t>(blockIdx.x) * KS_T + tid;
  const int G = gridDim.x;
  // The list is read-only during the sweep: the next atom's bounds and this
  // thread's first record of it are loaded ahead, while the current atom is
  // being processed.  A thread's first entry of the current atom (record and
  // residual row) stays in registers from phase 1 to phase 2.
  int lo = atom_start[0], hi = K > 0 ? atom_start[1] : 0;
  uint2 rec_next = lo + gtid < hi ? list[lo + gtid] : make_uint2(0u, 0u);
  for (int j = 0; j < K; ++j) {
    const uint2 rec0 = rec_next;
    const int nlo = hi;
    const int nhi = j + 2 <= K ? atom_start[j + 2] : hi;
    if (blockIdx.x == 0 && tid == 0) dead[j] = hi == lo ? 1 : 0;
    if (hi == lo) {
      if (blockIdx.x == 0 && tid < DLSH_D)
        D_new[static_cast<size_t>(j) * DLSH_D + tid] = D_old[static_cast<size_t>(j) * DLSH_D + tid];
      rec_next = nlo + gtid < nhi ? list[nlo + gtid] : make_uint2(0u, 0u);
      lo = nlo;
      hi = nhi;
      continue;  // the same decision in every CTA
    }
    if (tid < RROW) dj[tid] = tid < DLSH_D ? D_old[static_cast<size_t>(j) * DLSH_D + tid] : 0.f;
    // ---- phase 1: sum g R_i and g^2 over this thread's entries
    float v[64];
#pragma unroll
    for (int d = 0; d < 64; ++d) v[d] = 0.f;
    const bool has0 = lo + gtid < hi;
    const int64_t i0 = rec0.x & 0x3FFFFFFu;
    const float g0 = __uint_as_float(rec0.y);
    float4 r0[RROW / 4];
    if (has0) {
      const float4* r4 = reinterpret_cast<const float4*>(R + i0 * RROW);
#pragma unroll
      for (int q = 0; q < RROW / 4; ++q) r0[q] = __ldcg(r4 + q);
#pragma unroll
      for (int q = 0; q < RROW / 4; ++q) {
        if (4 * q + 0 < DLSH_D) v[4 * q + 0] = g0 * r0[q].x;
        if (4 * q + 1 < DLSH_D) v[4 * q + 1] = g0 * r0[q].y;
        if (4 * q + 2 < DLSH_D) v[4 * q + 2] = g0 * r0[q].z;
        if (4 * q + 3 < DLSH_D) v[4 * q + 3] = g0 * r0[q].w;
      }
      v[DLSH_D] = g0 * g0;  // after the row: slot 45 of the row is padding
    } else {
#pragma unroll
      for (int q = 0; q < RROW / 4; ++q) r0[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int64_t e = lo + gtid + gthreads; e < hi; e += gthreads) {
      const uint2 rec = list[e];
      const int64_t i = rec.x & 0x3FFFFFFu;
      const float g = __uint_as_float(rec.y);
      v[DLSH_D] = fmaf(g, g, v[DLSH_D]);
      const float4* r4 = reinterpret_cast<const float4*>(R + i * RROW);
#pragma unroll
      for (int q = 0; q < RROW / 4; ++q) {
        const float4 x = __ldcg(r4 + q);
        v[4 * q + 0] = fmaf(g, x.x, v[4 * q + 0]);
        v[4 * q + 1] = fmaf(g, x.y, v[4 * q + 1]);
        v[4 * q + 2] = fmaf(g, x.z, v[4 * q + 2]);
        if (4 * q + 3 < DLSH_D) v[4 * q + 3] = fmaf(g, x.w, v[4 * q + 3]);
      }
    }
    // transposing butterfly: after it, lane l holds the warp's sums of values
    // 2l and 2l + 1 in v[0], v[1]
#pragma unroll
    for (int m = 64, o = 16; o > 0; m >>= 1, o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int k = 0; k < m / 2; ++k) {
        const float send = up ? v[k] : v[k + m / 2];
        const float keep = up ? v[k + m / 2] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    wsum[warp][2 * lane] = v[0];
    wsum[warp][2 * lane + 1] = v[1];
    __syncthreads();
    if (tid < KS_V) {
      float sum = 0.f;
#pragma unroll
      for (int w = 0; w < KS_W; ++w) sum += wsum[w][tid];
      __stcg(part + static_cast<size_t>(blockIdx.x) * 48 + tid, sum);
    }
    if (!grid_barrier(gbar, budget, status)) return;
    rec_next = nlo + gtid < nhi ? list[nlo + gtid] : make_uint2(0u, 0u);
    // ---- phase 2: d = E^T g = sum g R_i + d_j sum g^2, in every CTA
    for (int f = tid; f < G * 48; f += KS_T) pall[f] = __ldcg(part + f);
    __syncthreads();
    if (tid < KS_V) {
      float sum = 0.f;
#pragma unroll 8
      for (int c = 0; c < G; ++c) sum += pall[c * 48 + tid];
      tot[tid] = sum;
    }
    __syncthreads();
    if (tid < 32) {
      const float v0 = fmaf(dj[tid], tot[DLSH_D], tot[tid]);
      const float v1 = tid < DLSH_D - 32 ? fmaf(dj[32 + tid], tot[DLSH_D], tot[32 + tid]) : 0.f;
      float n2 = fmaf(v0, v0, v1 * v1);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
      const bool zero = !(n2 > 0.f);
      const float inv = zero ? 0.f : rsqrtf(n2);
      const float u0 = v0 * inv, u1 = v1 * inv;
      dn[tid] = u0;
      if (tid < RROW - 32) dn[32 + tid] = u1;
      float dd = fmaf(dj[tid], u0, tid < DLSH_D - 32 ? dj[32 + tid] * u1 : 0.f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
      if (tid == 0) {
        dd_s = dd;
        skip_s = zero ? 1 : 0;
      }
      if (blockIdx.x == 0) {
        float* out = D_new + static_cast<size_t>(j) * DLSH_D;
        out[tid] = zero ? dj[tid] : u0;
        if (tid < DLSH_D - 32) out[32 + tid] = zero ? dj[32 + tid] : u1;
      }
    }
    __syncthreads();
    if (!skip_s) {
      const float dd = dd_s;
      const float4* dn4 = reinterpret_cast<const float4*>(dn);
      const float4* dj4 = reinterpret_cast<const float4*>(dj);
      if (has0) {
        // the first entry: record and row still in registers
        float e_dot = 0.f;
#pragma unroll
        for (int q = 0; q < RROW / 4; ++q) {
          const float4 u = dn4[q];
          e_dot = fmaf(r0[q].x, u.x, e_dot);
          e_dot = fmaf(r0[q].y, u.y, e_dot);
          e_dot = fmaf(r0[q].z, u.z, e_dot);
          e_dot = fmaf(r0[q].w, u.w, e_dot);
        }
        const float gn = fmaf(g0, dd, e_dot);
        float4* r4 = reinterpret_cast<float4*>(R + i0 * RROW);
#pragma unroll
        for (int q = 0; q < RROW / 4; ++q) {
          const float4 u = dn4[q], o = dj4[q];
          float4 y;
          y.x = fmaf(-gn, u.x, fmaf(g0, o.x, r0[q].x));
          y.y = fmaf(-gn, u.y, fmaf(g0, o.y, r0[q].y));
          y.z = fmaf(-gn, u.z, fmaf(g0, o.z, r0[q].z));
          y.w = fmaf(-gn, u.w, fmaf(g0, o.w, r0[q].w));
          __stcg(r4 + q, y);
        }
        coef[i0 * s + static_cast<int>(rec0.x >> 26)] = gn;
      }
      for (int64_t e = lo + gtid + gthreads; e < hi; e += gthreads) {
        const uint2 rec = list[e];
        const int64_t i = rec.x & 0x3FFFFFFu;
        const int slot = static_cast<int>(rec.x >> 26);
        const float g = __uint_as_float(rec.y);
        float4* r4 = reinterpret_cast<float4*>(R + i * RROW);
        float4 r[RROW / 4];
        float e_dot = 0.f;
#pragma unroll
        for (int q = 0; q < RROW / 4; ++q) {
          r[q] = __ldcg(r4 + q);
          const float4 u = dn4[q];
          e_dot = fmaf(r[q].x, u.x, e_dot);
          e_dot = fmaf(r[q].y, u.y, e_dot);
          e_dot = fmaf(r[q].z, u.z, e_dot);
          e_dot = fmaf(r[q].w, u.w, e_dot);  // padding: r = 0, u = 0
        }
        const float gn = fmaf(g, dd, e_dot);  // E_i . d = R_i . d + g (d_j . d)
#pragma unroll
        for (int q = 0; q < RROW / 4; ++q) {
          const float4 u = dn4[q], o = dj4[q];
          float4 y;
          y.x = fmaf(-gn, u.x, fmaf(g, o.x, r[q].x));
          y.y = fmaf(-gn, u.y, fmaf(g, o.y, r[q].y));
          y.z = fmaf(-gn, u.z, fmaf(g, o.z, r[q].z));
          y.w = fmaf(-gn, u.w, fmaf(g, o.w, r[q].w));
          __stcg(r4 + q, y);
        }
        coef[i * s + slot] = gn;
      }
    }
    if (!grid_barrier(gbar, budget, status)) return;
    lo = nlo;
    hi = nhi;
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
  if (N >= (int64_t(1) << 26))
    return set_error(DLSH_ERR_UNSUPPORTED,
                     "dlsh_mod_update: N must be < 2^26 (the atom lists pack signal and nnz in 32 bits)");
  Ws w;
  carve(ws, K, s, N, w);
  if (status_out) *status_out = w.status;
  size_t acc_smem = 0;
  const int acc_nw = accum_warps(K, s, &acc_smem);
  if (acc_nw == 0)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_mod_update: K=%d s=%d does not fit", K, s);
  DLSH_CUDA_TRY(cudaMemsetAsync(w.status, 0, sizeof(uint32_t), st), "dlsh_mod_update: reset");
  const int T = static_cast<int>((N + TS - 1) / TS > 0 ? (N + TS - 1) / TS : 1);
  int launches = 0;
  if (N > 0) {
    count_kernel<<<T, 256, K * sizeof(int), st>>>(idx, nnz, s, N, K, T, w.cnt, w.status);
  } else {
    DLSH_CUDA_TRY(cudaMemsetAsync(w.cnt, 0, sizeof(int) * K * T, st), "dlsh_mod_update: cnt");
  }
  atom_total_kernel<<<K, 256, 0, st>>>(w.cnt, T, w.atom_total);
  atom_scan_kernel<<<1, 1024, 0, st>>>(w.atom_total, K, w.atom_start);
  tile_offsets_kernel<<<K, 256, 0, st>>>(w.cnt, T, w.atom_start, w.off);
  launches += (N > 0 ? 1 : 0) + 3;
  if (N > 0) {
    const size_t sc_smem = scatter_smem(K, s);
    DLSH_CUDA_TRY(cudaFuncSetAttribute(scatter_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sc_smem)),
                  "dlsh_mod_update: attribute");
    scatter_kernel<false><<<T, SC_T, sc_smem, st>>>(idx, coef, nnz, s, N, K, T, w.off, w.list);
    ++launches;
  }
  void (*accum)(const float*, const uint16_t*, const float*, int, int, const int*, const int*, int, int, int,
                const int*, const uint2*, double*, double*) =
      s <= 8 ? accum_kernel<8> : (s <= 16 ? accum_kernel<16> : accum_kernel<32>);
  DLSH_CUDA_TRY(cudaFuncSetAttribute(accum, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(acc_smem)),
                "dlsh_mod_update: attribute");
  const int P = static_cast<int>(n_blocks(N));
  const int tpb = tiles_per_block(T);
  seg_scan_kernel<<<1, 1024, 0, st>>>(w.off, w.atom_start, T, tpb, K, P * K, w.seg_start);
  {
    int sms = device_sm_count();
    if (sms <= 0) sms = 1;
    int per_sm = 0;
    DLSH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, accum, acc_nw * 32, acc_smem),
                  "dlsh_mod_update: occupancy");
    if (per_sm < 1) per_sm = 1;
    int64_t grid = static_cast<int64_t>(sms) * per_sm;
    const int64_t ms = max_segments(K, s, N);
    if (grid > ms) grid = ms;
    accum<<<static_cast<int>(grid), acc_nw * 32, acc_smem, st>>>(X, idx, coef, s, K, w.atom_start, w.off, T, tpb,
                                                                 P * K, w.seg_start, w.list, w.Gp, w.Bp);
  }
  seg_reduce_kernel<<<K, 256, 0, st>>>(w.seg_start, w.Gp, w.Bp, K, P, w.M, w.Z);
  {
    const int nb = (K + MT - 1) / MT;
    mirror_kernel<<<dim3(nb, nb), MT * 8, 0, st>>>(w.M, K);
  }
  ridge_kernel<<<1, 1024, 0, st>>>(w.M, K, w.lam);
  launches += 5;
  // mixed-precision solve: FP32 Cholesky of the Jacobi-scaled matrix, then
  // kRefine FP32 solves with FP64 residuals in between
  scale_kernel<<<K, 256, 0, st>>>(w.M, w.Z, D_old, w.lam, K, w.dsc, w.A32, w.Zs, w.R32, w.Xs, w.Xb);
  ++launches;
  {
    static PerDevice<int> coop;
    int coop_grid = 0;
    const int crc = coop.get(&coop_grid, [](int& g) {
      int per_sm = 0;
      DLSH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_inv_kernel, CH_T, 0),
                    "dlsh_mod_update: occupancy");
      int sms = device_sm_count();
      if (sms <= 0) sms = 1;
      if (per_sm < 1) return set_error(DLSH_ERR_CUDA, "dlsh_mod_update: factorisation kernel does not fit");
      g = sms;  // one CTA per SM: fewer arrivals at each grid barrier
      return DLSH_OK;
    });
    if (crc) return crc;
    DLSH_CUDA_TRY(cudaMemsetAsync(w.gbar, 0, 2 * sizeof(unsigned), st), "dlsh_mod_update: barrier");
    float* A32 = w.A32;
    float* W32 = w.W32;
    int Kk = K;
    unsigned* gb = w.gbar;
    uint32_t* stw = w.status;
    long long budget = kWaitBudget;
    void* args[] = {&A32, &W32, &Kk, &gb, &stw, &budget};
    DLSH_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(chol_inv_kernel), dim3(coop_grid),
                                              dim3(CH_T), args, 0, st),
                  "dlsh_mod_update: factorisation");
    ++launches;
  }
  const int tr_grid = (K + 7) / 8;
  for (int it = 0; it < kRefine; ++it) {
    if (it > 0) {
      residual_kernel<<<(K + RS_ROWS - 1) / RS_ROWS, RS_T, 0, st>>>(w.M, w.lam, w.dsc, K, w.Zs, w.Xb, w.R32);
      ++launches;
    }
    trmm_kernel<false><<<tr_grid, 256, 0, st>>>(w.W32, K, w.R32, w.Y32, nullptr, nullptr, nullptr);
    trmm_kernel<true><<<tr_grid, 256, 0, st>>>(w.W32, K, w.Y32, nullptr, w.Xs, w.dsc, w.Xb);
    launches += 2;
  }
  normalise_kernel<<<(K + 7) / 8, 256, 0, st>>>(w.Xb, w.atom_start, K, D_new, D_old, w.dead);
  ++launches;
  if (resid && N > 0) {
    refill_kernel<<<1, 1024, 0, st>>>(X, resid, N, K, w.dead, D_new);
    ++launches;
  }
  count_launches(launches);
  return check_launch("dlsh_mod_update: launch");
}

size_t ksvd_ws_bytes(int K, int s, int64_t N) {
  mod::KsWs w;
  return mod::carve_ksvd(nullptr, K, s, N, w);
}

// Enqueues one approximate K-SVD sweep (no host synchronisation).
int ksvd_enqueue(const float* X, int64_t N, int K, const uint16_t* idx, float* coef, const uint8_t* nnz, int s,
                 const float* D_old, const float* resid, float* D_new, void* ws, cudaStream_t st,
                 uint32_t** status_out) {
  using namespace mod;
  if (N >= (int64_t(1) << 26))
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_ksvd_update: N must be < 2^26");
  KsWs w;
  carve_ksvd(ws, K, s, N, w);
  if (status_out) *status_out = w.status;
  DLSH_CUDA_TRY(cudaMemsetAsync(w.status, 0, sizeof(uint32_t), st), "dlsh_ksvd_update: reset");
  const int T = static_cast<int>((N + TS - 1) / TS > 0 ? (N + TS - 1) / TS : 1);
  int launches = 0;
  if (N > 0) {
    count_kernel<<<T, 256, K * sizeof(int), st>>>(idx, nnz, s, N, K, T, w.cnt, w.status);
  } else {
    DLSH_CUDA_TRY(cudaMemsetAsync(w.cnt, 0, sizeof(int) * K * T, st), "dlsh_ksvd_update: cnt");
  }
  atom_total_kernel<<<K, 256, 0, st>>>(w.cnt, T, w.atom_total);
  atom_scan_kernel<<<1, 1024, 0, st>>>(w.atom_total, K, w.atom_start);
  tile_offsets_kernel<<<K, 256, 0, st>>>(w.cnt, T, w.atom_start, w.off);
  launches += (N > 0 ? 1 : 0) + 3;
  if (N > 0) {
    const size_t sc_smem = scatter_smem(K, s);
    DLSH_CUDA_TRY(cudaFuncSetAttribute(scatter_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sc_smem)),
                  "dlsh_ksvd_update: attribute");
    scatter_kernel<true><<<T, SC_T, sc_smem, st>>>(idx, coef, nnz, s, N, K, T, w.off, w.list);
    ksvd_resid_kernel<<<static_cast<int>((N + 7) / 8), 256, 0, st>>>(X, D_old, K, idx, coef, nnz, s, N, w.R);
    launches += 2;
  }
  {
    static PerDevice<int> coop;
    int coop_grid = 0;
    const int crc = coop.get(&coop_grid, [](int& grid) {
      int per_sm = 0;
      int sms = device_sm_count();
      if (sms <= 0) sms = 1;
      const int g = sms < KS_MAX_GRID ? sms : KS_MAX_GRID;  // one CTA per SM
      const size_t sm_need = static_cast<size_t>(g) * 48 * sizeof(float);
      DLSH_CUDA_TRY(cudaFuncSetAttribute(ksvd_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm_need)),
                    "dlsh_ksvd_update: attribute");
      DLSH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ksvd_sweep_kernel, KS_T, sm_need),
                    "dlsh_ksvd_update: occupancy");
      if (per_sm < 1) return set_error(DLSH_ERR_CUDA, "dlsh_ksvd_update: sweep kernel does not fit");
      grid = g;
      return DLSH_OK;
    });
    if (crc) return crc;
    const size_t smem = static_cast<size_t>(coop_grid) * 48 * sizeof(float);
    DLSH_CUDA_TRY(cudaMemsetAsync(w.gbar, 0, 2 * sizeof(unsigned), st), "dlsh_ksvd_update: barrier");
    const int* as = w.atom_start;
    const uint2* li = w.list;
    int Kk = K, ss = s;
    float* cf = coef;
    const float* Do = D_old;
    float* Dn = D_new;
    float* Rr = w.R;
    float* pt = w.part;
    int* dd = w.dead;
    unsigned* gb = w.gbar;
    uint32_t* stw = w.status;
    long long budget = kWaitBudget;
    void* args[] = {&as, &li, &Kk, &ss, &cf, &Do, &Dn, &Rr, &pt, &dd, &gb, &stw, &budget};
    DLSH_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(ksvd_sweep_kernel), dim3(coop_grid),
                                              dim3(KS_T), args, smem, st),
                  "dlsh_ksvd_update: sweep");
    ++launches;
  }
  if (resid && N > 0) {
    refill_kernel<<<1, 1024, 0, st>>>(X, resid, N, K, w.dead, D_new);
    ++launches;
  }
  count_launches(launches);
  return check_launch("dlsh_ksvd_update: launch");
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
  if (reinterpret_cast<uintptr_t>(idx) % 4 != 0)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_mod_update: idx must be 4-byte aligned");
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

size_t dlsh_ksvd_workspace_size(int K, int d, int s, int64_t N) {
  if (d != DLSH_D || K < 1 || K > dlsh::mod::MAX_K || s < 1 || s > DLSH_MAX_S || N < 0) return 0;
  return dlsh::ksvd_ws_bytes(K, s, N);
}

int dlsh_ksvd_update(const float* X, int64_t N, int d, int K, const uint16_t* idx, float* coef,
                     const uint8_t* nnz, int s, const float* D_old, const float* resid_sq, float* D_new,
                     void* ws, size_t ws_bytes, void* stream, int flags) {
  using namespace dlsh;
  clear_error();
  if (d != DLSH_D) return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_ksvd_update: d must be 45");
  if (K < 1 || K > mod::MAX_K)
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_ksvd_update: K must be in [1, 4096], got %d", K);
  if (s < 1 || s > DLSH_MAX_S) return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_ksvd_update: s must be in [1, 32]");
  if (N < 0 || N * s >= (1LL << 31))
    return set_error(DLSH_ERR_UNSUPPORTED, "dlsh_ksvd_update: N*s must be < 2^31");
  if (!D_old || !D_new) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_ksvd_update: NULL D");
  if (D_old == D_new) return set_error(DLSH_ERR_INVALID_ARG, "dlsh_ksvd_update: D_new must not alias D_old");
  if (reinterpret_cast<uintptr_t>(idx) % 4 != 0)
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_ksvd_update: idx must be 4-byte aligned");
  if (N > 0 && (!X || !idx || !coef || !nnz))
    return set_error(DLSH_ERR_INVALID_ARG, "dlsh_ksvd_update: NULL array");
  int rc = check_workspace(ws, ws_bytes, ksvd_ws_bytes(K, s, N), "dlsh_ksvd_update");
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* status = nullptr;
  rc = ksvd_enqueue(X, N, K, idx, coef, nnz, s, D_old, resid_sq, D_new, ws, st, &status);
  if (rc) return rc;
  return finish(st, status, flags, "dlsh_ksvd_update");
}

}  // extern "C"
