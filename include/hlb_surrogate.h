/*
 * hlb_surrogate.h - C ABI of the sweep surrogate's training and inference
 * kernels (sm_103a, FP32).  The paper has no learned component; this network
 * serves the project's boiling-curve sweep (Section 4.4, Fig. 11 of arXiv
 * 1812.10375): from the superheat, the site count and the early wall-heat-flux
 * history of a run it predicts the run's quasi-steady mean wall heat flux and
 * a boiling-regime label, so that sweep points can be stopped early.
 *
 * Network (sizes from hlb_sur_config):
 *   x (B, 1, L0) -> conv1d(K, stride S) + ReLU -> (B, C1, L1)
 *                -> conv1d(K, S) + ReLU        -> (B, C2, L2)
 *                -> conv1d(K, S) + ReLU        -> (B, C3, L3) -> mean over time (B, C3)
 *   concat scalars (B, NS) -> linear H + ReLU -> linear H + ReLU -> linear NOUT.
 * Output 0 regresses the target; outputs 1..NOUT-1 are class logits.
 * Loss = mean (y0 - t)^2 + mean softmax cross-entropy of the logits.
 * Convolutions are unpadded: L_out = (L_in - K) / S + 1.
 *
 * Parameters are one flat FP32 vector in the order W1 (C1,1,K), b1,
 * W2 (C2,C1,K), b2, W3 (C3,C2,K), b3, F1 (H, C3+NS), c1, F2 (H,H), c2,
 * F3 (NOUT,H), c3, each row-major.  Inputs: hist (B, L0) row-major, scal
 * (B, NS), target (B), label (B, int32 in [0, NOUT-1)).
 *
 * All pointers are device pointers owned by the caller; d_ws is a device
 * workspace of hlb_sur_workspace_bytes(cfg, B) bytes (256-byte aligned) that
 * holds the activations between the forward and backward passes.  Calls are
 * asynchronous on `stream` (cudaStream_t as void*).  Errors: HLB_EINVAL for
 * bad sizes or pointers, HLB_ECUDA if a launch fails.
 */
#ifndef HLB_SURROGATE_H
#define HLB_SURROGATE_H

#include <stddef.h>

#include "hlb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int L0, C1, C2, C3, K, S, NS, H, NOUT;
} hlb_sur_config;

/* The default sizes: L0 = 500, channels 16/32/32, K = 5, S = 2, NS = 2, H = 256, NOUT = 6. */
void hlb_sur_config_default(hlb_sur_config* c);

/* Number of FP32 parameters; 0 for an invalid configuration. */
size_t hlb_sur_param_count(const hlb_sur_config* c);

/* Workspace bytes for a batch of B samples (1 <= B <= 4096). */
size_t hlb_sur_workspace_bytes(const hlb_sur_config* c, int B);

/* Forward pass: d_out (B, NOUT). */
hlb_status hlb_sur_forward(const hlb_sur_config* c, const float* d_params, const float* d_hist, const float* d_scal,
                           int B, float* d_out, void* d_ws, size_t ws_bytes, void* stream);

/* Forward + loss + backward: d_grad (same layout as the parameters) receives
 * dLoss/dparams; d_loss[0] = MSE term, d_loss[1] = cross-entropy term. */
hlb_status hlb_sur_loss_grad(const hlb_sur_config* c, const float* d_params, const float* d_hist,
                             const float* d_scal, const float* d_target, const int* d_label, int B, float* d_grad,
                             float* d_loss, void* d_ws, size_t ws_bytes, void* stream);

/* One bias-corrected Adam update (Kingma & Ba) of n parameters at step t >= 1. */
hlb_status hlb_sur_adam(long long n, float* d_params, const float* d_grad, float* d_m, float* d_v, float lr,
                        float beta1, float beta2, float eps, int t, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HLB_SURROGATE_H */
