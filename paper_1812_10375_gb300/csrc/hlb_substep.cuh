// Energy sub-steps of Eq. (27) for N > 1: the fused step kernel advances the
// flow and the first of the N RK4 sub-steps of the energy equation (its dt is
// already 1/N); the remaining N - 1 sub-steps run here, on the density and
// velocity of that LB step (rho^n, u^n, held fixed over the sub-steps as in
// the method: the flow moves once per LB step, the temperature N times).
//
// k_energy_substep: one RK4 sub-step (Eq. 18, dt = 1/N) of Eq. (17) with the
//   finite-volume diffusion of Eqs. (22)-(26), evaluated tile by tile with the
//   same arithmetic as the fused kernel's pass C and stages: a 56 x 24 tile in a
//   64 x 32 shared-memory frame (ring 4: stage k is evaluated on ring 4 - k).
//   It accumulates, per block, the RK-weighted wall fluxes of the sub-step and,
//   on the last sub-step, the sensible energy sum rho cv T of its cells.
// k_substep_fix: adds those fluxes to the diagnostics record that the step's
//   reduction wrote from the first sub-step, replaces its energy sum, and
//   corrects the running flux sum and the step's flux-history entry.
#pragma once
#include "hlb_kernels.cuh"

namespace hlb {

constexpr int SUB_TX = 56, SUB_TY = 24, SUB_H = 4;
constexpr int SUB_FW = SUB_TX + 2 * SUB_H;  // 64 frame columns, one per thread
constexpr int SUB_FH = SUB_TY + 2 * SUB_H;  // 32 frame rows
constexpr int SUB_NT = 256;
constexpr int SUB_NPH = SUB_NT / SUB_FW;  // 4 row phases
constexpr int SUB_NJ = SUB_FH / SUB_NPH;  // 8 frame rows per thread
constexpr int SUB_FN = SUB_FW * SUB_FH;
constexpr int SUB_NARR = 11;
constexpr size_t sub_smem_bytes() { return (size_t)SUB_NARR * SUB_FN * sizeof(float); }
static_assert(SUB_FW == 64 && SUB_NT % SUB_FW == 0 && SUB_FH % SUB_NPH == 0, "sub-step frame mapping");

// per-block partials of the sub-steps
enum { SP_QB = 0, SP_QT, SP_QI, SP_E, NSUBPART };

__global__ void __launch_bounds__(SUB_NT) k_energy_substep(const StepArgs A, const float* __restrict__ rho_n,
                                                           const float* __restrict__ ux_n,
                                                           const float* __restrict__ uy_n,
                                                           const float* __restrict__ T_in, float* __restrict__ T_out,
                                                           double* __restrict__ part, int first, int last) {
  extern __shared__ float sm[];
  float* const sT0 = sm;
  float* const sTa = sm + SUB_FN;
  float* const sTb = sm + 2 * SUB_FN;
  float* const sRho = sm + 3 * SUB_FN;
  float* const sUx = sm + 4 * SUB_FN;
  float* const sUy = sm + 5 * SUB_FN;
  float* const sLae = sm + 6 * SUB_FN;  // east-face conductivity (Eq. 25)
  float* const sLan = sm + 7 * SUB_FN;  // north-face conductivity
  float* const sIrcv = sm + 8 * SUB_FN;
  float* const sAs = sm + 9 * SUB_FN;   // latent-heat source coefficients
  float* const sBs = sm + 10 * SUB_FN;
  __shared__ double s_red[SUB_NT / 32][NSUBPART];
  __shared__ int s_err;

  const Geo g = make_geo(A);
  const int nx = A.nx, ny = A.ny;
  const int x0 = blockIdx.x * SUB_TX, y0 = blockIdx.y * SUB_TY;
  const int tid = threadIdx.x;
  const int i = tid % SUB_FW, jp = tid / SUB_FW;
  const int gxu = x0 - SUB_H + i;
  const int gx = wrapx(gxu, nx);
  const bool own_col = i >= SUB_H && i < SUB_H + SUB_TX && gxu < nx;
  const float lam_w = A.lambda_w, cvk = A.cvk;
  auto wall_lam = [&](int row) -> float { return g.top_wall && row == ny - 1 ? A.lambda_top : lam_w; };
  if (tid == 0) s_err = 0;
  int err = 0;

  // ---- load T (the wall value on Dirichlet rows), rho^n and u^n; frame rows
  // above the lattice copy row ny - 1 (the zero-gradient ghost of an open top),
  // rows below it are never read
#pragma unroll
  for (int m = 0; m < SUB_NJ; ++m) {
    const int j = jp + SUB_NPH * m;
    const int gy = y0 - SUB_H + j;
    const int idx = j * SUB_FW + i;
    if (gy < 0) {
      sT0[idx] = sRho[idx] = sUx[idx] = sUy[idx] = 0.f;
      continue;
    }
    const int gr = gy < ny ? gy : ny - 1;
    const long long c = (long long)gr * nx + gx;
    sT0[idx] = g.dirichlet_row(gr) ? (gr == 0 ? A.T_bottom : A.T_top) : T_in[c];
    sRho[idx] = rho_n[c];
    sUx[idx] = ux_n[c];
    sUy[idx] = uy_n[c];
  }
  __syncthreads();

  // ---- face conductivities on the whole frame; the other coefficients on
  // ring 3 (rows and columns 1 .. 62), as the fused kernel's pass C
#pragma unroll
  for (int m = 0; m < SUB_NJ; ++m) {
    const int j = jp + SUB_NPH * m;
    const int gy = y0 - SUB_H + j;
    if (gy < 0) continue;
    const int idx = j * SUB_FW + i;
    const int gr = gy < ny ? gy : ny - 1;
    const bool solid = g.solid_row(gr);
    const float lam = solid ? wall_lam(gr) : sRho[idx] * cvk;
    if (i + 1 < SUB_FW) {
      const float le = solid ? wall_lam(gr) : sRho[idx + 1] * cvk;
      sLae[idx] = 2.f * lam * le / (lam + le);
    }
    if (j + 1 < SUB_FH) {
      const int gn = gy + 1 < ny ? gy + 1 : ny - 1;
      const float ln = g.solid_row(gn) ? wall_lam(gn) : sRho[idx + SUB_FW] * cvk;
      sLan[idx] = 2.f * lam * ln / (lam + ln);
    }
    if (j < 1 || j >= SUB_FH - 1 || i < 1 || i >= SUB_FW - 1 || gy >= ny) continue;
    if (solid) {
      sIrcv[idx] = A.inv_rcv_w;
      sAs[idx] = 0.f;
      sBs[idx] = 0.f;
      continue;
    }
    const int js = j - 1, jn = j + 1;
    const float rho = sRho[idx];
    const float ircv = 1.f / (rho * A.cv);
    // div u with the isotropic gradient of Eq. (19)
    const float dux = (sUx[idx + 1] - sUx[idx - 1]) * (1.f / 3.f) +
                      ((sUx[jn * SUB_FW + i + 1] - sUx[js * SUB_FW + i - 1]) +
                       (sUx[js * SUB_FW + i + 1] - sUx[jn * SUB_FW + i - 1])) *
                          (1.f / 12.f);
    const float duy = (sUy[jn * SUB_FW + i] - sUy[js * SUB_FW + i]) * (1.f / 3.f) +
                      ((sUy[jn * SUB_FW + i + 1] - sUy[js * SUB_FW + i - 1]) +
                       (sUy[jn * SUB_FW + i - 1] - sUy[js * SUB_FW + i + 1])) *
                          (1.f / 12.f);
    const float divu = dux + duy;
    const float br = A.b * rho;
    // T (dp/dT)_rho = As' T + Bs' (1 + kappa (1 - sqrt Tr)) sqrt Tr (Eq. 28)
    const float Ar = rho * A.R / (1.f - br);
    const float Br = A.a * rho * rho * A.kappa / (1.f + 2.f * br - br * br);
    sIrcv[idx] = ircv;
    sAs[idx] = Ar * ircv * divu;
    sBs[idx] = Br * ircv * divu;
  }
  __syncthreads();

  // ---- RK4 stages (Eq. 18): stage k on ring 4 - k
  const int jtop = ny - 1 - y0 + SUB_H;  // frame row of the lattice's top row
  const bool has_ghost = jtop < SUB_FH - 1;
  const float dt = A.dt;
  float acc[SUB_NJ];
  double dq[3] = {0.0, 0.0, 0.0}, de = 0.0;
#pragma unroll
  for (int m = 0; m < SUB_NJ; ++m) acc[m] = 0.f;
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    const float* Tc = k == 1 ? sT0 : (k == 3 ? sTb : sTa);
    float* Tn = k == 1 ? sTa : (k == 2 ? sTb : sTa);
    const float cnext = k == 3 ? dt : 0.5f * dt;
    const float wk = (k == 1 || k == 4) ? dt * (1.f / 6.f) : dt * (2.f / 6.f);
    const float wacc = (k == 1) ? 1.f : 2.f;
    const int r = 4 - k;
    const bool col_in = i >= SUB_H - r && i < SUB_H + SUB_TX + r;
#pragma unroll
    for (int m = 0; m < SUB_NJ; ++m) {
      const int j = jp + SUB_NPH * m;
      const int gy = y0 - SUB_H + j;
      if (!col_in || j < SUB_H - r || j >= SUB_H + SUB_TY + r || gy < 0 || gy >= ny) continue;
      const bool own = own_col && j >= SUB_H && j < SUB_H + SUB_TY;
      const int idx = j * SUB_FW + i;
      const int js = j - 1, jn = j + 1;
      const float Tp = Tc[idx];
      float hk = 0.f;
      // row 0 under an imposed flux (Section 3.3): q_in enters through its bottom face
      const bool bot = gy == 0;
      if (!g.dirichlet_row(gy)) {
        const float TE = Tc[idx + 1], TW = Tc[idx - 1], TN = Tc[jn * SUB_FW + i], TS = Tc[js * SUB_FW + i];
        // Eqs. (22)-(26): the sum of the face fluxes of the control volume
        float kk = sLae[idx] * (TE - Tp);
        kk = fmaf(sLae[idx - 1], TW - Tp, kk);
        kk = fmaf(sLan[idx], TN - Tp, kk);
        kk = bot ? kk + A.q_in : fmaf(sLan[js * SUB_FW + i], TS - Tp, kk);
        kk *= sIrcv[idx];
        if (!g.solid_row(gy)) {
          const float TNE = Tc[jn * SUB_FW + i + 1], TNW = Tc[jn * SUB_FW + i - 1];
          const float TSE = Tc[js * SUB_FW + i + 1], TSW = Tc[js * SUB_FW + i - 1];
          const float gxT = (TE - TW) * (1.f / 3.f) + ((TNE - TSW) + (TSE - TNW)) * (1.f / 12.f);
          const float gyT = (TN - TS) * (1.f / 3.f) + ((TNE - TSW) + (TNW - TSE)) * (1.f / 12.f);
          kk -= sUx[idx] * gxT + sUy[idx] * gyT;
          const float sTr = sqrtf(fmaxf(Tp, 0.f) * A.invTc);
          kk -= sAs[idx] * Tp + sBs[idx] * (1.f + A.kappa * (1.f - sTr)) * sTr;
        }
        hk = kk;
      }
      if (k < 4) acc[m] += wacc * hk;
      if (own) {
        if (gy == 1) dq[0] += (double)(wk * sLan[js * SUB_FW + i] * (Tc[js * SUB_FW + i] - Tp));
        if (g.top_wall && gy == ny - 2) dq[1] += (double)(wk * sLan[idx] * (Tp - Tc[jn * SUB_FW + i]));
        if (gy == A.W) dq[2] += (double)(wk * sLan[js * SUB_FW + i] * (Tc[js * SUB_FW + i] - Tp));
        if (k == 4) {
          const float Tnew = sT0[idx] + dt * (1.f / 6.f) * (acc[m] + hk);
          if (nonfinite(Tnew)) err |= ERR_NONFINITE;
          T_out[(long long)gy * nx + gx] = Tnew;
          if (last) de += (double)(Tnew / sIrcv[idx]);
        }
      }
      if (k < 4) Tn[idx] = sT0[idx] + cnext * hk;
    }
    __syncthreads();
    if (k < 4 && has_ghost) {
      for (int j = jtop + 1 + jp; j < SUB_FH; j += SUB_NPH) Tn[j * SUB_FW + i] = Tn[jtop * SUB_FW + i];
      __syncthreads();
    }
  }

  // ---- per-block partials in FP64 (this path is not the hot one)
  double v[NSUBPART] = {dq[0], dq[1], dq[2], de};
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < NSUBPART; ++q) {
    const double s = warp_sum(v[q]);
    if (lane == 0) s_red[warp][q] = s;
  }
  if (err) atomicOr(&s_err, err);
  __syncthreads();
  if (tid < NSUBPART) {
    double s = 0.0;
    for (int w = 0; w < SUB_NT / 32; ++w) s += s_red[w][tid];
    double* p = part + (long long)(blockIdx.y * gridDim.x + blockIdx.x) * NSUBPART + tid;
    *p = first ? s : *p + s;
  }
  if (tid == 0 && s_err) atomicOr(&A.state->error_flags, s_err);
}

// Folds the sub-steps' partials into the diagnostics record of the step (one CTA).
__global__ void __launch_bounds__(256) k_substep_fix(const double* __restrict__ part, int nblk, DevState* st,
                                                      double inv_nx, double* hist) {
  __shared__ double s_red[8][NSUBPART];
  double v[NSUBPART] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NSUBPART; ++q) v[q] += part[(long long)b * NSUBPART + q];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NSUBPART; ++q) {
    const double s = warp_sum(v[q]);
    if (lane == 0) s_red[warp][q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[NSUBPART];
#pragma unroll
    for (int q = 0; q < NSUBPART; ++q) {
      s[q] = 0.0;
      for (int w = 0; w < 8; ++w) s[q] += s_red[w][q];
    }
    const double dqb = s[SP_QB] * inv_nx;
    st->q_bottom += dqb;
    st->q_top += s[SP_QT] * inv_nx;
    st->q_interface += s[SP_QI] * inv_nx;
    st->q_sum += dqb;
    st->energy = s[SP_E];
    // the reduction appended this step's first-sub-step flux unless the history was full
    if (hist && st->hist_len > 0 && st->hist_len == st->step) hist[st->hist_len - 1] = st->q_bottom;
  }
}

}  // namespace hlb
