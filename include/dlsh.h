/*
 * dlsh.h - C ABI of the GB300 sparse spherical-harmonic codec for 3D Gaussian
 * Splatting ("Smaller and Faster 3DGS via Post-Training Dictionary Learning").
 *
 * The codec replaces the 45 non-DC SH coefficients of every Gaussian (15 basis
 * functions of degree 1..3, times R, G, B) by a shared dictionary D and a sparse
 * code per Gaussian (Sec. 2.2).  D is learned by alternating minimisation of
 * Eq. 1 (codes by OMP, then the dictionary with the codes fixed, Sec. 2.1), and
 * radiance is evaluated straight from the sparse codes (Sec. 2.2).
 *
 * Conventions shared by every call
 *   - Signals x_i are d = 45 floats, channel-major: x[c*15 + b], c in {R,G,B},
 *     b = SH basis index 0..14 (l*l + l + m - 1 for degree l = 1..3, m = -l..l,
 *     real SH with the Condon-Shortley phase).
 *   - X is N x d row-major FP32.  The dictionary is passed as K x d row-major
 *     FP32: row j is atom j (the paper's D is its transpose, d x K).
 *   - Sparse codes use a padded ELL layout: idx[N*s] (uint16, atom indices in
 *     selection order, pad 0), coef[N*s] (FP32, pad 0), nnz[N] (uint8).
 *   - Every array argument is a caller-owned DEVICE pointer unless stated
 *     otherwise.  Pointers must be 16-byte aligned where the call says so.
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream) and returns a status code.  Argument
 *     errors are found on the host before anything is launched.  Device-side
 *     failures (a bounded wait that ran out, a bad value found by a kernel) are
 *     recorded in a status word inside the workspace; with DLSH_FLAG_SYNC the
 *     call synchronises the stream and turns that word into its return code.
 *   - Scratch memory: calls that need scratch take a caller-allocated workspace
 *     (`ws`, `ws_bytes`, 256-byte aligned) whose size the matching
 *     *_workspace_size() function returns.  The library itself never calls
 *     cudaMalloc.
 *   - On error, dlsh_last_error() returns a message for the calling thread.
 */
#ifndef DLSH_H
#define DLSH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define DLSH_OK               0
#define DLSH_ERR_INVALID_ARG (-1) /* null/misaligned pointer, bad size        */
#define DLSH_ERR_UNSUPPORTED (-2) /* d != 45, K > 65535, s > 32, ...          */
#define DLSH_ERR_CUDA        (-3) /* a CUDA runtime call failed               */
#define DLSH_ERR_TIMEOUT     (-4) /* a device-side bounded wait ran out       */
#define DLSH_ERR_WORKSPACE   (-5) /* workspace missing or too small           */
#define DLSH_ERR_DEVICE      (-6) /* a kernel flagged invalid data            */

/* ---- correlation precision of the OMP atom selection (D^T r) --------- */
#define DLSH_PREC_FP32 0 /* "plain FP32": each operand split into a high and a
                            low part of 11 significant bits and D^T r taken as
                            hi.hi + hi.lo + lo.hi on tcgen05 with FP32
                            accumulation (about 22 significant bits).  The
                            encoder for s <= 8 splits into FP16 parts of a
                            power-of-two scaled copy (the residual per row,
                            D by 256) -- twice the tensor rate and half the
                            operand bytes of TF32 parts; so does the one-tile
                            encoder for s > 8.  dlsh_correlate and the kernels
                            chosen by tuning records 3, 4, 64, 128 split into
                            TF32 parts                                      */
#define DLSH_PREC_BF16 1 /* BF16 operands, FP32 accumulate; each row's exact
                            low-precision top 4 (|c| truncated below the bits
                            that carry the column, then the smaller atom index)
                            is re-scored in FP32 before the commit              */
#define DLSH_PREC_FP8  2 /* E4M3 with per-atom and per-row scales; top 4
                            re-scored in FP32 as for BF16                        */
#define DLSH_PREC_BF16_QW 3 /* BF16 with a cheaper candidate set: the best atom of
                            each column quarter (j mod 128 in [32q, 32q+32)),
                            re-scored in FP32                                    */
#define DLSH_PREC_FP8_QW  4 /* FP8 with the column-quarter winners               */

/* ---- flags ------------------------------------------------------------ */
#define DLSH_FLAG_SYNC 1 /* synchronise the stream and report device status */

/* ---- limits ----------------------------------------------------------- */
#define DLSH_D      45    /* signal length (15 SH basis functions x RGB)      */
#define DLSH_MAX_K  65535 /* atom indices are stored as uint16                */
#define DLSH_MAX_S  32    /* maximum nonzeros per code                        */

/* Message describing the last error on the calling thread ("" if none). */
const char* dlsh_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
int dlsh_version(void);

/* Number of streaming multiprocessors of the current device (0 on failure). */
int dlsh_num_sms(void);

/* Running count of kernels this library has enqueued in this process (kernels
 * captured into a CUDA graph are counted once, at capture). */
unsigned long long dlsh_kernel_launches(void);

/*
 * Sparse coding by OMP (Sec. 2.1): for every signal x_i, greedily select up to s
 * atoms, each time the one of largest |d_j^T r| over atoms not yet selected
 * (ties: smallest j), then re-fit all selected coefficients by least squares,
 * r = x - D_I gamma.  Stops early when ||r||_2 <= eps (checked before each
 * selection), when max |d_j^T r| <= 1e-7 ||x||, or when the new atom is
 * numerically dependent on the selected ones (Cholesky pivot^2 <= 1e-6).
 *
 * D [K*d] FP32, X [N*d] FP32 (16-byte aligned), d must be 45, 1 <= K <= 65535,
 * 1 <= s <= 16, N >= 0.
 * Outputs: idx [N*s], coef [N*s], nnz [N], resid_sq [N] (||r||^2; may be NULL).
 * Workspace: dlsh_encode_workspace_size(K, d, s, precision) bytes.
 */
size_t dlsh_encode_workspace_size(int K, int d, int s, int precision);
int dlsh_encode(const float* D, int K, int d, const float* X, int64_t N, int s,
                float eps, int precision, uint16_t* idx, float* coef,
                uint8_t* nnz, float* resid_sq, void* ws, size_t ws_bytes,
                void* stream, int flags);

/*
 * The encoder kernel dlsh_encode runs for (K, s, precision) with the built-in
 * choice (no tuning record): 1 one tile per CTA, 2 two tiles on two warp
 * groups, 3 two tiles served in turn, 4 / 5 two tiles with selection and solver
 * warps (TF32 / FP16 parts), 6 three such tiles (FP16 parts), 7 one tile per
 * CTA with FP16 parts; 0 if the configuration is unsupported.  A record
 * from dlsh_autotune_encode overrides this choice.
 */
int dlsh_encode_variant(int K, int s, int precision);

/*
 * dlsh_encode with per-phase timing: identical results, plus twelve counters in
 * `cycles` (device, uint64[12], zeroed by the call) summed over all CTAs, in SM
 * clock cycles; counter 11 names the kernel that ran (1 one tile per CTA, 3 two
 * tiles served in turn, 4 / 5 / 6 selection and solver warps; the one-tile
 * kernel with FP16 parts reports 1).  The call
 * runs the kernel dlsh_encode would run, except that BF16/FP8 use the one-tile
 * kernel.  One tile (1): from the first selection/solver thread, waiting for the
 * tensor cores, the selection phase (including that wait), the barrier after
 * selection, the solver phase, the barrier after the solver, and the number of
 * OMP iterations counted; from the MMA-issuing thread, waiting for the A
 * operand (the residual), for a dictionary chunk to land, and for a TMEM buffer
 * to be released; from the TMA-producing thread, waiting for a free ring stage.
 * Two tiles in turn (3): selection waiting for the tensor cores, selection
 * (including that wait), solver, solver waiting for the staging area, tile
 * iterations, 0, then from the MMA thread: waiting for a residual, for a
 * dictionary chunk, for an accumulator buffer, and for the copy of the residual
 * into tensor memory.  Selection and solver warps (4): selection waiting for the
 * tensor cores, selection per job (including its waits), solver per job
 * (including its waits), solver waiting for the staging area, jobs, solver
 * waiting for candidates, the four MMA-thread counters as for (3), and
 * selection waiting for the solver to take its previous candidates (5 as 4).
 */
int dlsh_encode_profile(const float* D, int K, int d, const float* X, int64_t N,
                        int s, float eps, int precision, uint16_t* idx,
                        float* coef, uint8_t* nnz, float* resid_sq, void* ws,
                        size_t ws_bytes, unsigned long long* cycles, void* stream,
                        int flags);

/*
 * dlsh_encode without a workspace and without any allocation.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory, such
 * as plugins whose host application owns every device allocation through its
 * own pool, or real-time loops where a cudaMalloc (which may synchronise the
 * device) is not allowed.  Same arguments, outputs and stop rules as
 * dlsh_encode, minus `ws`/`ws_bytes`.
 *
 * Scratch lives in one fixed device array of dlsh_encode_noalloc_max_bytes()
 * bytes (8 MiB), which every GPU that loads the library holds until the process
 * exits; that covers K <= 1024 at every precision and s.  A configuration that
 * needs more returns DLSH_ERR_UNSUPPORTED before anything is launched.  A call
 * made while `stream` is not capturing looks up the array's device address on
 * the current device (so a context rebuilt after cudaDeviceReset is followed);
 * a call made while it is capturing uses the address from the device's last
 * lookup, and returns DLSH_ERR_INVALID_ARG if there was none.  All calls share
 * the array: calls whose work overlaps on the GPU (different streams, or
 * different host threads) race on it and must be serialised by the caller.
 */
size_t dlsh_encode_noalloc_max_bytes(void);
int dlsh_encode_noalloc(const float* D, int K, int d, const float* X, int64_t N,
                        int s, float eps, int precision, uint16_t* idx,
                        float* coef, uint8_t* nnz, float* resid_sq,
                        void* stream, int flags);

/*
 * Correlation step alone (the D^T r of every OMP iteration, Sec. 2.1) on the
 * same tensor-core path the encoder uses: C [M*K] = R [M*d] * D^T, FP32 result,
 * computed at `precision` (FP32 = 3xTF32; BF16; FP8 returns the scaled value
 * rho_i sigma_j (q_r . q_d)).  M >= 0.  Workspace: dlsh_encode_workspace_size.
 */
int dlsh_correlate(const float* D, int K, int d, const float* R, int64_t M,
                   int precision, float* C, void* ws, size_t ws_bytes,
                   void* stream, int flags);

/*
 * Radiance straight from the sparse codes (Sec. 2.2): for Gaussian i with view
 * direction v_i,  rgb_c = sum_{b} Y_b(v_i) * sum_{t < nnz_i} coef[i,t] * D[idx[i,t], c*15+b].
 * If cam_pos (HOST pointer to 3 floats) is NULL, dirs_or_means [N*3] holds unit
 * view directions; otherwise it holds Gaussian means mu_i and
 * v_i = (mu_i - cam) / ||mu_i - cam||.  Output rgb [N*3] FP32.  With dc NULL
 * the output is the view-dependent part only (the DC term is not part of the
 * dictionary); with dc [N*3] (device, the DC SH coefficient of each channel)
 * it is the full colour max(0, Y00 dc + view-dependent part + 0.5),
 * Y00 = 1/(2 sqrt(pi)).  No workspace.
 */
int dlsh_decode(const float* D, int K, int d, const uint16_t* idx,
                const float* coef, const uint8_t* nnz, int s, int64_t N,
                const float* dirs_or_means, const float* cam_pos, const float* dc,
                float* rgb, void* stream, int flags);

/*
 * Dictionary update with the codes fixed (the second half of the alternating
 * minimisation of Eq. 1), read as MOD:
 *   G = A A^T, B = X A^T, lambda = 1e-6 trace(G)/K (1e-6 if trace is 0),
 *   D~ = (B + lambda D_old)(G + lambda I)^-1, solved on the device with an FP32
 *   Cholesky factor of the Jacobi-scaled matrix and FP64 iterative refinement
 *   (G and B accumulated in float-float: about FP64 accuracy),
 *   d_j = d~_j / ||d~_j||; atoms with no nonzero in A (or d~_j = 0) are
 *   refilled in increasing j with the normalised signals of largest resid_sq
 *   (decreasing order, ties to the smallest index, zero signals skipped).
 * D_old, D_new [K*d]; resid_sq [N] (needed only when an atom is unused; may be
 * NULL, then unused atoms keep D_old).  Accumulation order is fixed: results
 * are bitwise reproducible.  Limits: K <= 4096, N < 2^26, N*s < 2^31
 * (DLSH_ERR_UNSUPPORTED otherwise).  Workspace: dlsh_mod_workspace_size(K, d, s, N).
 */
size_t dlsh_mod_workspace_size(int K, int d, int s, int64_t N);
int dlsh_mod_update(const float* X, int64_t N, int d, int K,
                    const uint16_t* idx, const float* coef, const uint8_t* nnz,
                    int s, const float* D_old, const float* resid_sq,
                    float* D_new, void* ws, size_t ws_bytes, void* stream,
                    int flags);

/*
 * Alternating minimisation of Eq. 1 (Sec. 2.1): D_0 = normalised X rows at
 * init_idx [K] (int64, distinct, device), then `iters` times
 * {codes = OMP(D, X); D = MOD(D, codes)} and a final OMP pass.  Writes the final
 * dictionary D_out [K*d], the final codes, and rmse [iters+1] (device FP32,
 * sqrt(sum ||r||^2 / (N d)) after every coding pass).  The whole loop is
 * captured once into a CUDA graph and replayed; no host synchronisation happens
 * inside it.  Workspace: dlsh_learn_workspace_size(...).
 */
/*
 * First step of the learning loop alone: D_out row j = X[init_idx[j]] /
 * ||X[init_idx[j]]||, init_idx [K] int64 on the device (the random choice of
 * signals is an input).  Rows whose index is out of range or whose signal is
 * zero are left unwritten.  No workspace.
 */
int dlsh_init_dictionary(const float* X, int64_t N, int d, const int64_t* init_idx,
                         int K, float* D_out, void* stream, int flags);

size_t dlsh_learn_workspace_size(int K, int d, int s, int64_t N, int precision);
int dlsh_learn_dictionary(const float* X, int64_t N, int d, int K, int s,
                          float eps, int iters, const int64_t* init_idx,
                          int precision, float* D_out, uint16_t* idx,
                          float* coef, uint8_t* nnz, float* rmse, void* ws,
                          size_t ws_bytes, void* stream, int flags);

/* ---- many scenes in one call ---------------------------------------------
 * Several independent encoding problems (one per scene: its own dictionary D,
 * K, signals X [N x 45], s and eps; outputs as in dlsh_encode) in one call.
 * Each scene is encoded exactly as dlsh_encode would encode it (same plan, so
 * bitwise the same codes), on internal streams forked from `stream` and joined
 * back to it: scenes run concurrently, the most expensive (N*K*s) first.
 * precision: FP32, BF16 or FP8 for every scene; bn: 0 (tuned/default), a
 * kernel variant of every scene (2..7 as dlsh_encode_variant numbers them;
 * 64 / 128: one tile with that atom-chunk width), plus optionally 256 x a cap
 * of 2..32 on the dictionary ring's stages (fewer stages than fit; the codes
 * do not depend on it).  Invalid bn: DLSH_ERR_INVALID_ARG.  At most 32 scenes,
 * s <= 16; scenes with N = 0 are skipped.  The call enqueues only kernels and
 * event record/wait (no host copies), so it can be captured into a CUDA graph;
 * the scene table is read at enqueue time.  Workspace: see
 * dlsh_encode_multi_workspace_size (0 = invalid scene table). */
typedef struct dlsh_scene {
  const float* D;   /* K x 45 */
  int K;
  const float* X;   /* N x 45 */
  int64_t N;
  int s;
  float eps;
  uint16_t* idx;    /* N x s */
  float* coef;      /* N x s */
  uint8_t* nnz;     /* N */
  float* resid_sq;  /* N, may be NULL */
} dlsh_scene;
size_t dlsh_encode_multi_workspace_size(const dlsh_scene* scenes, int n, int precision, int bn);
int dlsh_encode_multi(const dlsh_scene* scenes, int n, int precision, int bn, void* ws,
                      size_t ws_bytes, void* stream, int flags);

/* Autotuner: times dlsh_encode on the caller's sample with every encoder kernel
 * whose plan fits (variants 2..7 of dlsh_encode_variant, and one tile with 64
 * or 128 atoms per MMA), each with as many dictionary ring stages as fit; then,
 * for the fastest, half that many stages and the kernel's minimum (2; 3 for
 * variant 2).  It records the fastest (kernel, stages) for (K, s, precision),
 * and later dlsh_encode / dlsh_encode_multi calls use it.  *best_bn (host, may
 * be NULL) = the kernel (low byte) + 256 x the stage cap (0: as many as fit).
 * With DLSH_AUTOTUNE_CACHE set to a file path the table of tuned choices
 * (encoder and decode) is kept there as JSON lines and read back at first use.
 * Outputs are scratch of the sample's size.  On an error no trial choice stays
 * recorded. */
int dlsh_autotune_encode(const float* D, int K, int d, const float* X, int64_t N, int s,
                         int precision, uint16_t* idx, float* coef, uint8_t* nnz,
                         float* resid_sq, void* ws, size_t ws_bytes, void* stream, int* best_bn);

/* The encoder choice recorded for (K, s, precision) by dlsh_autotune_encode in
 * this process or read from DLSH_AUTOTUNE_CACHE: the kernel (low byte) + 256 x
 * the ring-stage cap, as *best_bn reports it; 0 if none is recorded or the
 * arguments are out of range.  Host only (no GPU work). */
int dlsh_tuned_encode(int K, int s, int precision);

/* ---- learned support proposal ------------------------------------------
 * An extension of the paper's plain OMP (Sec. 2.1): a 45 -> 256 -> 256 -> K MLP
 *   xn = x/||x|| (0 if x = 0); h1 = gelu(W1 xn + b1); h2 = gelu(W2 h1 + b2);
 *   z = W3 h2 + b3;  gelu(u) = u Phi(u) (exact erf form)
 * trained with mean BCE-with-logits against the multi-hot OMP support and Adam
 * (beta 0.9/0.999, eps 1e-8, FP32 master weights, BF16 weights in every GEMM,
 * FP32 accumulation on tcgen05).  Its 2s largest logits (ties: smaller index)
 * are the candidates of an OMP restricted to them; plain OMP is the fallback.
 *
 * Parameters live in a caller-owned blob of dlsh_mlp_size(K) bytes (256-byte
 * aligned).  The parameter vector (dlsh_mlp_num_params(K) floats) is, in order:
 * W1 [256 x 64] (input padded from 45 to 64; columns 45..63 are zero), b1
 * [256], W2 [256 x 256], b2 [256], W3 [K x 256], b3 [K], all row-major. */
long long dlsh_mlp_num_params(int K);
size_t dlsh_mlp_size(int K);
/* Batch workspace for forward / gradients / training with batches of B rows. */
size_t dlsh_mlp_workspace_size(int K, int64_t B);
/* Sets the parameters from `params` (device FP32) and zeroes the Adam state. */
int dlsh_mlp_init(void* mlp, int K, const float* params, void* stream, int flags);
/* Copies the FP32 parameter vector out (device). */
int dlsh_mlp_params(const void* mlp, int K, float* params, void* stream, int flags);
/* Logits [B x K] of the signals X [B x 45], by the fused inference kernel of
 * dlsh_mlp_propose (the layer-by-layer training forward gives the same bits). */
int dlsh_mlp_forward(const void* mlp, int K, const float* X, int64_t B, float* logits,
                     void* ws, size_t ws_bytes, void* stream, int flags);
/* Gradients of the mean BCE loss (layout of the parameter vector) for the
 * targets given as ELL supports (idx [B x s], nnz [B]); loss (device, 1). */
int dlsh_mlp_gradients(const void* mlp, int K, const float* X, int64_t B,
                       const uint16_t* idx, const uint8_t* nnz, int s, float* grads,
                       float* loss, void* ws, size_t ws_bytes, void* stream, int flags);
/* One Adam step (step counts from 1) on one batch. */
int dlsh_mlp_train_step(void* mlp, int K, const float* X, int64_t B, const uint16_t* idx,
                        const uint8_t* nnz, int s, float lr, int64_t step, float* loss,
                        void* ws, size_t ws_bytes, void* stream, int flags);
/* `epochs` passes over N signals in consecutive batches (N / batch per epoch),
 * learning rate lr * (1 + cos(pi t / T)) / 2; loss_per_step (device, may be
 * NULL) receives every step's loss.  Workspace: dlsh_mlp_workspace_size(K, batch). */
int dlsh_mlp_train(void* mlp, int K, const float* X, int64_t N, const uint16_t* idx,
                   const uint8_t* nnz, int s, int epochs, int64_t batch, float lr,
                   float* loss_per_step, void* ws, size_t ws_bytes, void* stream, int flags);
/* The m (2, 4, 8, 16 or 32) largest logits of every signal, largest first,
 * equal logits by smaller atom index: cand [N x m] uint16 atom indices (0xFFFF
 * where K < m leaves a slot empty).  One fused kernel computes the three layers
 * and the selection on chip, with the arithmetic of dlsh_mlp_forward, so cand
 * is exactly the top m of that call's logits.  cand must be aligned to
 * min(16, 2m) bytes and ws to 256 bytes (else DLSH_ERR_INVALID_ARG); the
 * workspace size depends on K only. */
size_t dlsh_mlp_propose_workspace_size(int K, int64_t N);
int dlsh_mlp_propose(const void* mlp, int K, const float* X, int64_t N, int m,
                     uint16_t* cand, void* ws, size_t ws_bytes, void* stream, int flags);
/* OMP restricted to each signal's m candidate atoms (s <= m <= 32): the same
 * greedy steps, stop rules and outputs as dlsh_encode, the argmax taken over the
 * candidates only (ties: smaller atom index).  Workspace:
 * dlsh_encode_workspace_size(K, d, s, DLSH_PREC_FP32). */
int dlsh_encode_restricted(const float* D, int K, int d, const float* X, int64_t N,
                           const uint16_t* cand, int m, int s, float eps, uint16_t* idx,
                           float* coef, uint8_t* nnz, float* resid_sq, void* ws,
                           size_t ws_bytes, void* stream, int flags);
/* Learned encoder: MLP proposal of m candidates (m = 0: 2s; otherwise one of
 * 2, 4, 8, 16, 32 with s <= m), restricted OMP, and plain OMP (at
 * fallback_precision, any DLSH_PREC_*) as the fallback.  mode 0 ("exact"): plain OMP runs on
 * every signal and replaces the learned code when ||r_learned|| > ||r_plain|| *
 * (1 + 1e-6).  mode 1 ("deploy"): plain OMP runs only on the signals with
 * ||r_learned|| > tau.  n_fallback (device, uint64) receives the count. */
size_t dlsh_encode_learned_workspace_size(int K, int d, int s, int64_t N, int m);
int dlsh_encode_learned(const float* D, int K, int d, const float* X, int64_t N, int s,
                        float eps, const void* mlp, int m, int mode, float tau,
                        int fallback_precision, uint16_t* idx, float* coef, uint8_t* nnz,
                        float* resid_sq, unsigned long long* n_fallback, void* ws,
                        size_t ws_bytes, void* stream, int flags);
/* Deploy-mode threshold from a calibration set: the tau whose fallback set is
 * the smallest that keeps sqrt(sum r) within max_ratio of plain OMP's, given
 * both residual vectors (device); *tau is written on the host. */
int dlsh_calibrate_fallback(const float* resid_learned, const float* resid_plain, int64_t N,
                            float max_ratio, float* tau, void* stream);

/*
 * Compact code storage (the paper stores each Gaussian's nonzeros and their
 * indices, Sec. 2.2; here at reduced width): FP16 coefficients and 8-bit atom
 * indices when K <= 256 (else 16-bit), nnz unchanged.
 * dlsh_compact_codes converts ELL codes (idx [N x s] uint16, coef [N x s] FP32)
 * to that form: idx_out [N x s] of idx_bytes (1 or 2) each, coef_out [N x s]
 * IEEE FP16 bits (round to nearest).  DLSH_ERR_UNSUPPORTED when idx_bytes = 1
 * and K > 256.
 * dlsh_decode_compact is dlsh_decode on compact codes: the FP32 dictionary D
 * is rounded to FP16 as it is staged in shared memory (128 bytes per atom, the
 * three channels of a basis in one 8-byte word); sums are FP32.  K must not
 * exceed dlsh_decode_compact_max_k(s) (the shared-memory dictionary, about
 * 1600 atoms), else DLSH_ERR_UNSUPPORTED.  The result differs from dlsh_decode
 * by the FP16 rounding of D and of the coefficients only.
 */
size_t dlsh_decode_compact_max_k(int s);
int dlsh_compact_codes(const uint16_t* idx, const float* coef, int64_t N, int s, int K,
                       void* idx_out, int idx_bytes, uint16_t* coef_out, void* stream, int flags);
int dlsh_decode_compact(const float* D, int K, int d, const void* idx, int idx_bytes,
                        const uint16_t* coef_f16, const uint8_t* nnz, int s, int64_t N,
                        const float* dirs_or_means, const float* cam_pos, const float* dc,
                        float* rgb, void* stream, int flags);

/* Decode autotuner: times the decode of the caller's codes with batches of 8
 * and of 16 Gaussians per warp, each at three warp counts per CTA (as many as
 * fit beside the shared-memory dictionary, three quarters and half of that;
 * 32, 24 and 16 where rows are read through the read-only cache), and records
 * the fastest for (format, K, s); later dlsh_decode / dlsh_decode_compact calls
 * of that shape use it.  The colours do not depend on the choice.
 *   format 0: dlsh_decode's codes (idx uint16, coef FP32);
 *          1 / 2: compact codes with 8- / 16-bit indices and FP16 coef.
 * rgb (N x 3, device) is scratch; the DC term is not applied.  *best_batch and
 * *best_warps: host, may be NULL.  Errors: d != 45, s outside [1, 32] or K
 * outside the format's range -> DLSH_ERR_UNSUPPORTED; format outside 0..2,
 * N < 1 or a NULL array -> DLSH_ERR_INVALID_ARG (both before any GPU work). */
int dlsh_autotune_decode(const float* D, int K, int d, const void* idx, const void* coef, int format,
                         const uint8_t* nnz, int s, int64_t N, const float* dirs_or_means,
                         const float* cam_pos, float* rgb, void* stream, int* best_batch,
                         int* best_warps);

/* The decode shape recorded for (format, K, s), format as in
 * dlsh_autotune_decode: returns 1 and sets *batch and *warps (host, may be
 * NULL) if one is recorded, else 0 (also for arguments out of range).  A
 * record that no longer fits beside the dictionary is ignored by the decode.
 * Host only (no GPU work). */
int dlsh_tuned_decode(int format, int K, int s, int* batch, int* warps);

/*
 * The paper's storage format (Sec. 2.2): the code matrix A (K x N) in
 * Compressed Sparse Column form, one column per Gaussian.  col_ptr [N+1]
 * (int64), row_idx and val have room for N*s entries; col_ptr[N] = total nnz.
 * Workspace: dlsh_csc_workspace_size(N).
 */
size_t dlsh_csc_workspace_size(int64_t N);
int dlsh_csc_from_ell(const uint16_t* idx, const float* coef,
                      const uint8_t* nnz, int64_t N, int s, int64_t* col_ptr,
                      uint16_t* row_idx, float* val, void* ws, size_t ws_bytes,
                      void* stream, int flags);

/*
 * Dictionary update read as approximate K-SVD (an alternative to MOD under the
 * same alternating minimisation of Eq. 1, Sec. 2.1; one power step per atom as
 * in Rubinstein, Zibulevsky and Elad, 2008).  A sweep over j = 0..K-1 in order:
 * with w the Gaussians whose first nnz code slots hold atom j, g their current
 * coefficients of atom j, and R = X - D A the current residual,
 *   E = R_w + g d_j^T,  d = E^T g / ||E^T g||,  g' = E d,
 *   d_j <- d,  A[j, w] <- g',  R_w <- E - g' d^T.
 * An atom whose d is zero is left as it was; atoms no code uses are refilled,
 * in increasing j, with the normalised signals of largest resid_sq (as in
 * dlsh_mod_update; with resid_sq NULL they keep D_old).  The supports (idx,
 * nnz) are unchanged; coef [N*s] is updated IN PLACE.  Atom indices within a
 * code must be distinct (as the encoder writes them).  D_new [K*d] must not
 * alias D_old.  Every sum runs in a fixed order: results are bitwise
 * reproducible.  Limits: K <= 4096, N < 2^26, N*s < 2^31.  The sweep is one
 * cooperative launch with two bounded grid barriers per used atom.
 * Workspace: dlsh_ksvd_workspace_size(K, d, s, N) (it holds R: N*45 floats).
 */
size_t dlsh_ksvd_workspace_size(int K, int d, int s, int64_t N);
int dlsh_ksvd_update(const float* X, int64_t N, int d, int K, const uint16_t* idx, float* coef,
                     const uint8_t* nnz, int s, const float* D_old, const float* resid_sq,
                     float* D_new, void* ws, size_t ws_bytes, void* stream, int flags);

/* ---- splatting preprocess: project, cull, colour ----------------------------
 * The per-Gaussian preprocess of a Gaussian-splatting renderer, with the
 * colour step read either from dense SH (the baseline renderer) or from the
 * shared dictionary and each Gaussian's nonzeros (the paper's renderer,
 * Sec. 2.2).  With p_c = R mu + t (camera space, z forward):
 *   Sigma   = R(q) diag(scale)^2 R(q)^T, q = (w, x, y, z), normalised here;
 *   J       = [[fx/z, 0, -fx x'/z], [0, fy/z, -fy y'/z]], x' = clamp(x/z, +-1.3 W/(2 fx)),
 *             y' likewise with H and fy;
 *   S2      = (J R) Sigma (J R)^T + 0.3 I = [[a, b], [b, c]];
 *   xy      = (fx x/z + W/2, fy y/z + H/2), depth = z, conic = S2^-1 as (a', b', c');
 *   radius  = ceil(3 sqrt(mid + sqrt(max(0.1, mid^2 - det)))), mid = (a + c)/2;
 *   visible = z > z_near, det > 0, and the square of that radius meets the image;
 *   rgb     = max(0, Y00 dc + sum_b Y_b(v) y[c*15+b] + 0.5), Y00 = 1/(2 sqrt(pi)),
 *             v = (mu - C)/|mu - C|, C = -R^T t the camera centre,
 *             y the Gaussian's 45 SH coefficients or D^T alpha from its codes.
 * A culled Gaussian gets radius 0 and zeros in every other output; its colour
 * coefficients are not read.  All arrays are device memory, caller-owned;
 * cam, g and out are HOST pointers to the structs.  quats must be 16-byte and
 * xy 8-byte aligned.  Code entries with t >= nnz, or an index >= K, count as
 * zero (as in dlsh_decode).  No workspace.  Results are FP32. */
typedef struct dlsh_camera {
  float R[9];         /* world -> camera rotation, row-major */
  float t[3];         /* world -> camera translation */
  float fx, fy;       /* focal lengths in pixels (> 0) */
  int width, height;  /* image size in pixels; the principal point is its centre */
  float z_near;       /* near plane */
} dlsh_camera;

typedef struct dlsh_gaussians {
  const float* means;   /* [N*3] world positions */
  const float* scales;  /* [N*3] standard deviations along the local axes */
  const float* quats;   /* [N*4] rotations (w, x, y, z), nonzero */
  const float* dc;      /* [N*3] DC SH coefficient of each channel */
  int64_t N;
} dlsh_gaussians;

typedef struct dlsh_splat_out {
  float* xy;       /* [N*2] pixel centre */
  float* depth;    /* [N] camera-space z */
  float* conic;    /* [N*3] inverse screen covariance (a', b', c') */
  int32_t* radius; /* [N] pixels; 0 = culled */
  float* rgb;      /* [N*3] colour */
} dlsh_splat_out;

/* Colour from dense SH: sh [N*45], channel-major (c*15 + b). */
int dlsh_preprocess_sh(const dlsh_camera* cam, const dlsh_gaussians* g, const float* sh,
                       const dlsh_splat_out* out, void* stream, int flags);
/* Colour from ELL codes (idx [N*s] u16, coef [N*s] FP32, nnz [N]) and the FP32
 * dictionary D [K*45], held in shared memory: K <= dlsh_preprocess_max_k(s, 0),
 * else DLSH_ERR_UNSUPPORTED. */
int dlsh_preprocess_codes(const dlsh_camera* cam, const dlsh_gaussians* g, const float* D, int K,
                          const uint16_t* idx, const float* coef, const uint8_t* nnz, int s,
                          const dlsh_splat_out* out, void* stream, int flags);
/* Colour from compact codes (the dlsh_compact_codes format); D is rounded to
 * FP16 in shared memory as in dlsh_decode_compact; K <= dlsh_preprocess_max_k(s, 1). */
int dlsh_preprocess_compact(const dlsh_camera* cam, const dlsh_gaussians* g, const float* D, int K,
                            const void* idx, int idx_bytes, const uint16_t* coef_f16,
                            const uint8_t* nnz, int s, const dlsh_splat_out* out, void* stream,
                            int flags);
/* Largest K the shared-memory dictionary of the codes (compact = 0) or compact
 * (compact = 1) preprocess holds at sparsity s; 0 for an invalid s. */
size_t dlsh_preprocess_max_k(int s, int compact);

/* ---- self-test of the bounded device waits --------------------------------
 * Not part of the method (the paper has no counterpart): every pipelined kernel
 * here waits on mbarriers or a grid barrier with a cycle budget, so that a lost
 * arrival ends in DLSH_ERR_TIMEOUT instead of a hung GPU.  This call makes such
 * a wait run out on purpose, with nothing else in flight: kind 0 waits on an
 * mbarrier nobody arrives on; kind 1 is a cooperative launch in which one CTA
 * skips the grid barrier.  budget_cycles (1 .. 4e9 SM cycles) bounds the wait.
 * Returns DLSH_ERR_TIMEOUT when the wait gave up as designed; the CUDA context
 * stays usable.  ws: dlsh_selftest_workspace_size() bytes of device memory,
 * 256-byte aligned.  Synchronises the stream. */
size_t dlsh_selftest_workspace_size(void);
int dlsh_selftest_bounded_wait(int kind, int64_t budget_cycles, void* ws, size_t ws_bytes,
                               void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DLSH_H */
