// Enqueue-only entry points shared between the library's translation units.
// None of them synchronises; each returns a DLSH_* status and leaves a device
// status word (OR of ST_* bits) where *status_out points.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace dlsh {

// Batch-OMP encoder (encode.cu).  bn = 0: the tuned or default atom-chunk
// width; 64 or 128 forces it (FP32 only).  n_dev: optional signal count read on
// the device (the launch then covers every SM).
int encode_enqueue(const float* D, int K, const float* X, int64_t N, int s, float eps, int prec,
                   uint16_t* idx, float* coef, uint8_t* nnz, float* resid_sq, void* ws,
                   cudaStream_t st, uint32_t** status_out, unsigned long long* prof = nullptr,
                   const long long* n_dev = nullptr, int bn = 0);
// Dictionary preparation only (padded FP32 copy and Gram matrix).
int encode_prepare_only(const float* D, int K, int s, int prec, void* ws, cudaStream_t st,
                        const float** D32p, const float** G, uint32_t** status);
// Workspace bytes of encode_enqueue (largest over the admissible widths).
size_t encode_ws_bytes(int K, int s, int prec);

// MOD dictionary update (mod.cu).
int mod_enqueue(const float* X, int64_t N, int K, const uint16_t* idx, const float* coef,
                const uint8_t* nnz, int s, const float* D_old, const float* resid, float* D_new,
                void* ws, cudaStream_t st, uint32_t** status_out);
size_t mod_ws_bytes(int K, int s, int64_t N);

// Support-proposal MLP (mlp.cu).
size_t mlp_train_ws_bytes(int K, long long B);

// Fused inference (propose.cu): the m highest-logit atoms of every signal, or
// (infer_logits_enqueue) the logits themselves, N x K.  The workspace
// (propose_ws_bytes, 256-byte aligned) holds the packed weights.
size_t propose_ws_bytes(int K);
int propose_enqueue(const void* mlp_blob, int K, const float* X, long long N, int m, uint16_t* cand,
                    void* ws, uint32_t* status, cudaStream_t st);
int infer_logits_enqueue(const void* mlp_blob, int K, const float* X, long long N, float* logits,
                         void* ws, uint32_t* status, cudaStream_t st);

}  // namespace dlsh
