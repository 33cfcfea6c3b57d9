// Internal device-side descriptors of the hybrid thermal LB step (arXiv 1812.10375).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hlb {

// Per-block FP64 partial sums written by the step kernel.
enum { P_MASS = 0, P_ENERGY, P_QB, P_QT, P_QI, P_UTOP, P_VCOV, NPART };

// Error word bits (match the header's description).
enum { ERR_NONFINITE = 1, ERR_PSI_NEG = 2, ERR_TIMEOUT = 4 };

// Device-resident scalars of one domain.  Written only by the reduction kernel
// (and atomically OR-ed error bits by the step kernel).
struct DevState {
  double rho_ave;       // fluid-mean density of the last step (used by the next, Eq. 9)
  double rho_ave_prev;  // the value the last step used
  double U;             // lagged convective-outlet velocity (>= 0)
  double Uc;            // U / (1 + U), formed in FP64 (keeps U's precision when U << 1)
  long long step;
  double mass, energy, q_bottom, q_top, q_interface, u_top;
  double q_sum;
  long long q_count;
  double vcov, vcov_sum;  // vapour fraction of the first fluid row, and its running sum
  int error_flags;
  int hist_len;
};

// Everything the fused step kernel needs, passed by value.
struct StepArgs {
  int nx, ny, W, top_bc, eos_T_fixed;
  long long plane;  // nx * ny
  // Peng-Robinson (Eq. 28)
  float R, a, b, kappa, invTc, Ts;
  // forces (Eqs. 6, 9, 10) and forcing (Eq. 8)
  float G, g_y;
  float sig_e, sig_z;  // (1 - s/2) * C * sigma / (tau - 1/2) for rows e and zeta
  // relaxation (Eq. 3)
  float s_e, s_z, s_j, s_q;
  float tau_l, tau_v, rho_v, dtau_drho;
  float rho_ref;  // deviation storage reference
  float rho_mid;  // (rho_l + rho_v) / 2: vapour below, liquid above
  // energy (Eq. 17)
  float cvk, cv, rcv_w, inv_rcv_w, lambda_w, dt;
  float lambda_top;  // conductivity of a top wall row
  int bottom_flux;   // row 0 heated by the imposed flux q_in instead of held at T_bottom
  float q_in;
  int iso;          // isotropic central diffusion (Eqs. 20-21) instead of the finite-volume faces
  float kd, kd_w;   // lambda / (rho cv) of the fluid (k) and of the solid
  float inv_k;      // 1 / k: rho cv of a fluid cell from its lambda
  float T_bottom, T_top;
  // buffers
  const float* __restrict__ f_in;
  float* __restrict__ f_out;
  const float* __restrict__ T_in;
  float* __restrict__ T_out;
  const float* __restrict__ Gw;
  const float* __restrict__ ftop_in;
  float* __restrict__ ftop_out;
  double* __restrict__ partials;
  DevState* state;
  // split step (flow kernel, then energy sub-steps): rho^n, u_x^n, u_y^n as three
  // planes of nx ny floats written by the flow kernel, a temperature plane for
  // sub-steps, and the per-tile partial sums of the two kernels
  float* __restrict__ mom;
  float* __restrict__ T_scr;
  double* __restrict__ fpart;
  double* __restrict__ epart;
};

// The per-domain part of StepArgs for the batched kernel (geometry, wall
// temperatures, buffers); the model parameters are shared by the batch and
// reach the kernel as a by-value argument.
struct DomArgs {
  int nx, ny, W, top_bc, eos_T_fixed;
  long long plane;
  float T_bottom, T_top;
  const float* f_in;
  float* f_out;
  const float* T_in;
  float* T_out;
  const float* Gw;
  const float* ftop_in;
  float* ftop_out;
  double* partials;
  DevState* state;
  float* mom;
  float* T_scr;
  double* fpart;
  double* epart;
};

// Asynchronous 4-byte global-to-shared copies (cp.async, .ca).  The kernels
// that use them copy into and later read only slots of their own thread, so
// cp.async.wait_group alone makes the data visible to the reader.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
// 16-byte form (both addresses 16-byte aligned; bypasses L1)
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// all but the N most recently committed groups of this thread complete
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace hlb
