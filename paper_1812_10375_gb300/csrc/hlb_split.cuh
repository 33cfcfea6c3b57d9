// Split form of the coupled step of the hybrid thermal LB phase-change model
// (Hu & Liu, arXiv 1812.10375): one step of a domain is a flow kernel, N
// energy sub-step kernels (Eq. 27) and the FP64 reduction.
//
// k_flow (one launch per step): pull-streaming with halfway bounce-back and the
//   open-top rules (Eqs. 1-2, Sections 3.3, 4.2) -> rho (Eq. 5) -> psi from the
//   Peng-Robinson EOS at T^n (Eqs. 7, 28) -> F = F_m + F_ads + F_b (Eqs. 6, 9,
//   10) -> u (Eq. 5) -> MRT collision with Li's forcing (Eqs. 2-4, 8).  It
//   writes the post-collision populations and rho^n, u^n for the energy update.
//   A tile is 64 columns by TY fluid rows; psi of its cells and of a one-cell
//   ring around it goes through shared memory (the ring's populations are
//   pulled again by this CTA, from L2).  Each thread keeps the pulled
//   populations of its own cells in registers between the psi pass and the
//   collision, so every population is loaded once and stored once.
// k_energy (N launches per step): one RK4 sub-step (Eq. 18, dt = 1/N) of the
//   energy equation (Eq. 17) with the finite-volume harmonic face
//   conductivities of Eqs. (22)-(26), on rho^n and u^n held over the
//   sub-steps.  A 56 x 24 tile in a 64 x 32 frame; stage k is evaluated on
//   ring 4 - k of the tile.  Each thread owns a run of 8 rows of one frame
//   column: the per-cell coefficients of Eq. (17) (four face terms with the
//   axis part of the advection folded in, two diagonal advection terms, the
//   two latent-heat coefficients, rho cv) and the run's stage values stay in
//   registers; shared memory carries only what neighbouring threads read (the
//   stage values, u and lambda).
// Both kernels write per-tile partial sums (flow: fluid mass, first-fluid-row
// vapour count, top outlet velocity; energy: RK-weighted wall fluxes over the
// sub-steps, sensible energy of T^{n+1}) that k_reduce_split folds into the
// device record in FP64.
//
// HBM bytes per fluid cell and step: populations 36 read + 36 written, T^n 4
// read and rho^n, u^n 12 written by the flow kernel; T 4 read + 4 written and
// rho^n, u^n 12 read by each energy sub-step.  108 B at N = 1 against the 80 B
// of the fused kernel, in exchange for a flow kernel without halo recompute
// beyond one ring and an energy kernel without the flow's ring-5 halo.
#pragma once
#include "hlb_kernels.cuh"

namespace hlb {

enum { FP_MASS = 0, FP_VCOV, FP_UTOP, NFPART };
enum { EP_QB = 0, EP_QT, EP_QI, EP_E, NEPART };

constexpr int FL_TX = 64;          // flow tile width
constexpr int FL_FW = FL_TX + 2;   // psi frame: the tile and a one-cell ring
// Compiled split-step variants: flow tile (fluid rows, threads per CTA, CTAs
// per SM) and energy layout (rows per thread run, runs, CTAs per SM).
// TYF, NTHF, MINBF: the flow tile's fluid rows, threads and CTAs per SM; RP:
// the flow kernel pulls its own cells again after the barrier instead of
// holding their populations in registers (fewer registers, more CTAs per SM).
// TILE(TYF, NTHF, MINBF, RP, R, NPH, MINB): the energy tile of R-row runs;
// WALK(TYF, NTHF, MINBF, RP, L, MINB, PF): the row-walking energy kernel over
// L-row segments, sized for MINB CTAs per SM, its input rows fetched PF rows
// ahead by asynchronous copies into shared memory (PF = 0: one row ahead into
// registers).
#define HLB_SPLIT_VARIANTS(TILE, WALK) \
  WALK(24, 256, 4, 1, 64, 10, 6) WALK(16, 256, 4, 1, 64, 10, 6) WALK(16, 256, 3, 0, 64, 10, 6) \
  WALK(16, 256, 3, 0, 96, 8, 4) WALK(16, 256, 3, 0, 96, 8, 0) TILE(16, 256, 3, 0, 8, 4, 2)

constexpr int EN_TX = 56, EN_TY = 24, EN_H = 4;
constexpr int EN_FW = EN_TX + 2 * EN_H;  // 64 frame columns, one per thread
constexpr int EN_FH = EN_TY + 2 * EN_H;  // 32 frame rows
constexpr int EN_FN = EN_FW * EN_FH;
constexpr int EN_NARR = 5;               // T^n, two stage buffers (one doubles as u_x), u_y, lambda
constexpr size_t energy_smem_bytes() { return (size_t)EN_NARR * EN_FN * sizeof(float); }
static_assert(EN_FW == 64, "energy frame mapping");
// Energy-kernel thread layouts over the 64 x 32 frame: rows per thread run R
// and runs NPH (R * NPH = 32 frame rows, 64 * NPH threads).

template <int TY>
constexpr size_t flow_smem_bytes() { return (size_t)FL_FW * (TY + 2) * sizeof(float); }

// The batch kernels' per-domain descriptor applied to the shared model parameters.
__device__ __forceinline__ void apply_dom(StepArgs& A, const DomArgs& D) {
  A.nx = D.nx;
  A.ny = D.ny;
  A.W = D.W;
  A.top_bc = D.top_bc;
  A.eos_T_fixed = D.eos_T_fixed;
  A.plane = D.plane;
  A.T_bottom = D.T_bottom;
  A.T_top = D.T_top;
  A.f_in = D.f_in;
  A.f_out = D.f_out;
  A.T_in = D.T_in;
  A.T_out = D.T_out;
  A.Gw = D.Gw;
  A.ftop_in = D.ftop_in;
  A.ftop_out = D.ftop_out;
  A.partials = D.partials;
  A.state = D.state;
  A.mom = D.mom;
  A.T_scr = D.T_scr;
  A.fpart = D.fpart;
  A.epart = D.epart;
}

// Rows of the flow grid: the fluid rows [W, fluid_end).
__host__ __device__ __forceinline__ int fluid_end(int ny, int top_bc) { return top_bc == 0 ? ny - 1 : ny; }

// A flow tile whose frame rows [y0 - 1, y0 + TY] lie in [W + 1, ny - 3]: every
// pull of its cells is plain streaming (no solid row within two rows, not the
// open top row) and none of its cells is a diagnostic or outlet row.
__device__ __forceinline__ bool flow_interior(const StepArgs& A, int y0, int TY) {
  return y0 - 1 >= A.W + 1 && y0 + TY <= A.ny - 3;
}

// Compensated block reduction of NQ per-thread (hi, lo) pairs into FP64 slots
// out[0..NQ) (one thread writes each; `add` adds to the stored value).
template <int NTH, int NQ>
__device__ __forceinline__ void block_partials(float (&ah)[NQ], float (&al)[NQ], float (*s_red)[NQ][2],
                                               double* out, bool add) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    if (__any_sync(0xffffffffu, ah[q] != 0.f || al[q] != 0.f)) ff_warp_sum(ah[q], al[q]);
    if (lane == 0) {
      s_red[warp][q][0] = ah[q];
      s_red[warp][q][1] = al[q];
    }
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    const int q = threadIdx.x;
    float hi = s_red[0][q][0], lo = s_red[0][q][1];
#pragma unroll
    for (int w = 1; w < NTH / 32; ++w) ff_merge(hi, lo, s_red[w][q][0], s_red[w][q][1]);
    const double v = (double)hi + (double)lo;
    out[q] = add ? out[q] + v : v;
  }
}

// ---------------------------------------------------------------- flow tile
template <int TY, int NTH, bool INT, bool RP>
__device__ __forceinline__ void flow_tile(const StepArgs& A, int bx, int by, int part, float* sPsi, float Uc,
                                          float rho_ave) {
  constexpr int NPH = NTH / FL_TX;
  constexpr int CPT = TY / NPH;  // own cells per thread: a run of CPT rows of one column
  constexpr int NHALO = 2 * FL_FW + 2 * TY;
  static_assert(NTH % FL_TX == 0 && TY % NPH == 0, "one thread per tile column and row run");
  __shared__ float s_red[NTH / 32][NFPART][2];
  __shared__ int s_err;

  const Geo g = make_geo(A);
  const int nx = A.nx, ny = A.ny, W = A.W;
  const int fend = g.top_wall ? ny - 1 : ny;
  const int x0 = bx * FL_TX, y0 = W + by * TY;
  const int tid = threadIdx.x;
  const int i = tid & (FL_TX - 1), jp = tid / FL_TX;
  const int gxu = x0 + i;
  const int gx = wrapx(gxu, nx);
  const int xm = gx == 0 ? nx - 1 : gx - 1;
  const int xp = gx == nx - 1 ? 0 : gx + 1;
  const bool colv = gxu < nx;
  const int P = (int)A.plane;
  const int NC = nx * ny;
  if (tid == 0) s_err = 0;
  int err = 0;

  // psi of a fluid node from its density and temperature (Eq. 7 with Eq. 28)
  auto psi_of = [&](float rho, float T) -> float {
    float p2 = pr_psi2(A, rho, A.eos_T_fixed ? A.Ts : T);
    if (!(p2 >= 0.f)) {
      err |= ERR_PSI_NEG;
      p2 = 0.f;
    }
    return sqrtf(p2);
  };
  // populations of fluid node (x, y) after streaming, with the wall and top rules
  auto pull_any = [&](int x, int y, float h[9]) {
    const int hxm = x == 0 ? nx - 1 : x - 1, hxp = x == nx - 1 ? 0 : x + 1;
    pull(A, g, x, hxm, hxp, y, y - 1 < W, g.top_wall && y + 1 == ny - 1, Uc, h);
  };

  // ---- pass 1: pull the tile's own cells (kept in registers), rho, psi
  const int o1 = P + xm - gx, o3 = 3 * P + xp - gx;
  const int o2 = 2 * P - nx, o5 = 5 * P - nx + xm - gx, o6 = 6 * P - nx + xp - gx;
  const int o4 = 4 * P + nx, o7 = 7 * P + nx + xp - gx, o8 = 8 * P + nx + xm - gx;
  // the pulled populations of own cell (gx, gy) into h
  auto own_pull = [&](int gy, float h[9]) {
    if (INT) {
      const float* __restrict__ F = A.f_in + gy * nx + gx;
      h[0] = __ldg(F);
      h[1] = __ldg(F + o1);
      h[3] = __ldg(F + o3);
      h[2] = __ldg(F + o2);
      h[5] = __ldg(F + o5);
      h[6] = __ldg(F + o6);
      h[4] = __ldg(F + o4);
      h[7] = __ldg(F + o7);
      h[8] = __ldg(F + o8);
    } else {
      pull(A, g, gx, xm, xp, gy, gy == W, g.top_wall && gy + 1 == ny - 1, Uc, h);
    }
  };
  // RP: pass 2 pulls the own cells again (from L1/L2) instead of keeping their
  // populations in registers across the barrier
  float f[RP ? 1 : CPT][9];
  float rho[CPT];
#pragma unroll
  for (int m = 0; m < CPT; ++m) {
    const int j = jp * CPT + m;
    const int gy = y0 + j;
    float ps = 0.f;
    rho[m] = 1.f;
    if (INT || gy < fend) {
      const int c = gy * nx + gx;
      float* fm = f[RP ? 0 : m];
      own_pull(gy, fm);
      rho[m] = A.rho_ref + sum9(fm);
      ps = psi_of(rho[m], __ldg(A.T_in + c));
    } else if (g.top_open && gy == ny) {
      // zero-gradient ghost above an open top: psi of row ny - 1
      float h[9];
      pull_any(gx, ny - 1, h);
      ps = psi_of(A.rho_ref + sum9(h), __ldg(A.T_in + (ny - 1) * nx + gx));
    }
    sPsi[(j + 1) * FL_FW + i + 1] = ps;
  }
  // ---- the ring: rows y0 - 1 and y0 + TY (all 66 frame columns), columns
  // x0 - 1 and x0 + 64 (the tile's rows); solid rows carry no psi
  for (int t = tid; t < NHALO; t += NTH) {
    int j, ii;
    if (t < 2 * FL_FW) {
      j = t < FL_FW ? -1 : TY;
      ii = (t < FL_FW ? t : t - FL_FW) - 1;
    } else {
      const int s = t - 2 * FL_FW;
      ii = s < TY ? -1 : FL_TX;
      j = s < TY ? s : s - TY;
    }
    int gy = y0 + j;
    if (g.top_open && gy == ny) gy = ny - 1;  // zero-gradient ghost
    float ps = 0.f;
    if (gy >= W && gy < fend) {
      const int hx = wrapx(x0 + ii, nx);
      float h[9];
      pull_any(hx, gy, h);
      ps = psi_of(A.rho_ref + sum9(h), __ldg(A.T_in + gy * nx + hx));
    }
    sPsi[(j + 1) * FL_FW + ii + 1] = ps;
  }
  __syncthreads();

  // ---- pass 2: forces, velocity, collision of the own cells
  float ah[NFPART], al[NFPART];
#pragma unroll
  for (int q = 0; q < NFPART; ++q) ah[q] = al[q] = 0.f;
  const float gw = __ldg(A.Gw + gx);
  // RP: one cell at a time (the loop is not unrolled, so the pulls of the next
  // cell are not hoisted), rho recomputed from the same pull and summation
#pragma unroll RP ? 1 : CPT
  for (int m = 0; m < CPT; ++m) {
    const int j = jp * CPT + m;
    const int gy = y0 + j;
    if (!colv || !(INT || gy < fend)) continue;
    const int idx = (j + 1) * FL_FW + i + 1;
    const float psi = sPsi[idx];
    if (RP) own_pull(gy, f[0]);
    const float r = RP ? A.rho_ref + sum9(f[0]) : rho[m];
    const bool sol_s = !INT && gy == W;
    const bool sol_n = !INT && g.top_wall && gy == ny - 2;
    // Eq. (6); a solid neighbour carries psi(x)
    const float pE = sPsi[idx + 1], pW = sPsi[idx - 1];
    const float pN = sol_n ? psi : sPsi[idx + FL_FW];
    const float pS = sol_s ? psi : sPsi[idx - FL_FW];
    const float pNE = sol_n ? psi : sPsi[idx + FL_FW + 1];
    const float pNW = sol_n ? psi : sPsi[idx + FL_FW - 1];
    const float pSE = sol_s ? psi : sPsi[idx - FL_FW + 1];
    const float pSW = sol_s ? psi : sPsi[idx - FL_FW - 1];
    const float sx = (pE - pW) * (1.f / 3.f) + ((pNE - pNW) + (pSE - pSW)) * (1.f / 12.f);
    const float sy = (pN - pS) * (1.f / 3.f) + ((pNE + pNW) - (pSE + pSW)) * (1.f / 12.f);
    const float Fmx = -A.G * psi * sx;
    const float Fmy = -A.G * psi * sy;
    // Eq. (10) with weights omega/3: only a normal component next to a solid row
    const float Fay = INT ? 0.f : gw * psi * psi * ((float)sol_n - (float)sol_s) * (1.f / 6.f);
    const float Fx = Fmx;
    const float Fy = Fmy + Fay + (r - rho_ave) * A.g_y;  // Eq. (9)
    const float* fm = f[RP ? 0 : m];
    // the collision's moment sums (the same expressions, computed once)
    const float jx = (fm[1] - fm[3]) + ((fm[5] - fm[7]) - (fm[6] - fm[8]));
    const float jy = (fm[2] - fm[4]) + ((fm[5] - fm[7]) + (fm[6] - fm[8]));
    const float irho = 1.f / r;
    const float ux = (jx + 0.5f * Fx) * irho;
    const float uy = (jy + 0.5f * Fy) * irho;
    const int c = gy * nx + gx;
    const float fsum = collide_store(A, fm, r, ux, uy, Fx, Fy, A.G * A.G * (sx * sx + sy * sy), c);
    if (nonfinite(fsum)) err |= ERR_NONFINITE;
    A.mom[c] = r;
    A.mom[NC + c] = ux;
    A.mom[2 * NC + c] = uy;
    ff_add(ah[FP_MASS], al[FP_MASS], r);
    if (!INT) {
      if (gy == W && r < A.rho_mid) ff_add(ah[FP_VCOV], al[FP_VCOV], 1.f);
      if (gy == ny - 2) ff_add(ah[FP_UTOP], al[FP_UTOP], uy);
      if (A.top_bc == TOP_CONVECTIVE && gy == ny - 1) {
        A.ftop_out[gx] = fm[4];
        A.ftop_out[nx + gx] = fm[7];
        A.ftop_out[2 * nx + gx] = fm[8];
      }
    }
  }
  if (err) atomicOr(&s_err, err);
  block_partials<NTH, NFPART>(ah, al, s_red, A.fpart + (long long)part * NFPART, false);
  if (tid == 0 && s_err) atomicOr(&A.state->error_flags, s_err);
}

template <int TY, int NTH, int MINB, bool RP>
__global__ void __launch_bounds__(NTH, MINB) k_flow(const StepArgs A) {
  extern __shared__ float sm[];
  const float Uc = (float)A.state->Uc, rho_ave = (float)A.state->rho_ave;
  const int part = blockIdx.y * gridDim.x + blockIdx.x;
  const int y0 = A.W + blockIdx.y * TY;
  if (flow_interior(A, y0, TY))
    flow_tile<TY, NTH, true, RP>(A, blockIdx.x, blockIdx.y, part, sm, Uc, rho_ave);
  else
    flow_tile<TY, NTH, false, RP>(A, blockIdx.x, blockIdx.y, part, sm, Uc, rho_ave);
}

// Loads the domain descriptor of block `b` into shared memory; returns false
// for a stopped domain.
template <int NTH>
__device__ __forceinline__ bool batch_prologue(const DomArgs* __restrict__ desc, const int2* __restrict__ blk,
                                               const int* __restrict__ active, const float2* __restrict__ lag,
                                               DomArgs& sD, int2& s_bl, float2& s_lg, int& s_act) {
  const int2 bl = blk[blockIdx.x];
  const int* src = reinterpret_cast<const int*>(desc + bl.x);
  int* dst = reinterpret_cast<int*>(&sD);
  for (int q = threadIdx.x; q < (int)(sizeof(DomArgs) / sizeof(int)); q += NTH) dst[q] = src[q];
  if (threadIdx.x == NTH - 1) {
    s_bl = bl;
    s_act = active[bl.x];
    s_lg = lag ? lag[bl.x] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  return s_act != 0;
}

// Batched flow step: block b takes tile blk[b].y of domain blk[b].x.
template <int TY, int NTH, int MINB, bool RP>
__global__ void __launch_bounds__(NTH, MINB) k_flow_batch(const StepArgs P, const DomArgs* __restrict__ desc,
                                                          const int2* __restrict__ blk,
                                                          const int* __restrict__ active,
                                                          const float2* __restrict__ lag) {
  extern __shared__ float sm[];
  __shared__ DomArgs sD;
  __shared__ int s_act;
  __shared__ int2 s_bl;
  __shared__ float2 s_lg;
  if (!batch_prologue<NTH>(desc, blk, active, lag, sD, s_bl, s_lg, s_act)) return;
  StepArgs A = P;
  apply_dom(A, sD);
  const int local = s_bl.y;
  const int tx = (A.nx + FL_TX - 1) / FL_TX;
  const int by = local / tx;
  if (flow_interior(A, A.W + by * TY, TY))
    flow_tile<TY, NTH, true, RP>(A, local % tx, by, local, sm, s_lg.x, s_lg.y);
  else
    flow_tile<TY, NTH, false, RP>(A, local % tx, by, local, sm, s_lg.x, s_lg.y);
}

// -------------------------------------------------------------- energy tile
// Temperature buffers of sub-step s of N: X_0 = T^n (T_in), X_N = T^{n+1}
// (T_out); the others alternate with the scratch plane so that X_N lands in T_out.
__device__ __forceinline__ float* substep_buffer(const StepArgs& A, int s, int nsub) {
  return ((nsub - s) & 1) ? A.T_scr : A.T_out;
}

// Harmonic mean of two conductivities (Eq. 25 with dx = 1).
__device__ __forceinline__ float harm(float a, float b) { return 2.f * a * b / (a + b); }

// Per-cell coefficients of the energy right-hand side K(T) of Eq. (17):
//   K = aE (T_E - T) + aW (T_W - T) + aN (T_N - T) + aS (T_S - T)
//       - p (T_NE - T_SW) - q (T_SE - T_NW) - As T - Bs s (1 + kappa - kappa s),
// s = sqrt(T / Tc).  The face terms are lambda_f / (rho cv) of Eqs. (22)-(26);
// the isotropic gradient of Eq. (19) in u . grad T contributes -u_x/3, +u_x/3,
// -u_y/3, +u_y/3 to them and p = (u_x + u_y)/12, q = (u_x - u_y)/12 on the
// diagonals; As, Bs are the latent-heat coefficients (T dp/dT)_rho div u /
// (rho cv) of Eq. (28) split into the T and the sqrt(T) parts.  Solid rows
// keep only the face terms; Dirichlet rows have all coefficients zero.
enum { C_AE = 0, C_AW, C_AN, C_AS, C_P, C_Q, C_AS_T, C_BS, NCOEF };

// An energy tile whose frame rows [y0 - 4, y0 + 28) all lie in [W, ny - 2]:
// no solid, Dirichlet, ghost or wall-flux row in the frame.
__device__ __forceinline__ bool energy_interior(const StepArgs& A, int y0) {
  return y0 - EN_H >= A.W && y0 + EN_TY + EN_H <= A.ny - 1;
}

// The same sub-step on an interior tile, without branches: every frame row of
// every run is evaluated in every stage (rows outside a stage's ring get
// values that nothing valid reads), and the coefficients use that
// lambda = rho cv k in the fluid: lambda_f / (rho cv) = 2 k lambda_nb /
// (lambda + lambda_nb), and the latent-heat coefficients need no 1/(rho cv).
template <int R, int NPH>
__device__ __forceinline__ void energy_tile_int(const StepArgs& A, int bx, int by, int part, float* sm, int s,
                                                int nsub) {
  constexpr int FW = EN_FW, H = EN_H, FH = R * NPH, TY = FH - 2 * H, FN = FW * FH, NT = FW * NPH;
  static_assert(TY == EN_TY && FH == EN_FH, "energy tile geometry");
  float* const sT = sm;
  float* const sA = sm + FN;
  float* const sB = sm + 2 * FN;
  float* const sUy = sm + 3 * FN;
  float* const sLam = sm + 4 * FN;
  float* const sUx = sB;
  __shared__ float s_red[NT / 32][NEPART][2];
  __shared__ int s_err;

  const float* __restrict__ T_in = s == 1 ? A.T_in : substep_buffer(A, s - 1, nsub);
  float* __restrict__ T_out = substep_buffer(A, s, nsub);
  const bool last = s == nsub;
  const int nx = A.nx, ny = A.ny;
  const int NC = nx * ny;
  const float* __restrict__ rho_n = A.mom;
  const float* __restrict__ ux_n = A.mom + NC;
  const float* __restrict__ uy_n = A.mom + 2 * NC;
  const int x0 = bx * EN_TX, y0 = by * TY;
  const int tid = threadIdx.x;
  const int i = tid & (FW - 1), jp = tid / FW;
  const int j0 = jp * R;
  const int gy0 = y0 - H + j0;
  const int gxu = x0 - H + i;
  const int gx = wrapx(gxu, nx);
  const bool own_col = i >= H && i < H + EN_TX && gxu < nx;
  const int ie = i + 1 < FW ? i + 1 : i, iw = i > 0 ? i - 1 : i;  // frame-edge columns read themselves
  if (tid == 0) s_err = 0;
  int err = 0;

  // ---- load T^n, rho^n, u^n; lambda = rho cv k
  float T0[R], rho[R], lam[R];
  const float* tp = T_in + gy0 * nx + gx;
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int o = m * nx;
    const float T = __ldg(tp + o);
    rho[m] = __ldg(rho_n + (tp - T_in) + o);
    const float ux = __ldg(ux_n + (tp - T_in) + o);
    const float uy = __ldg(uy_n + (tp - T_in) + o);
    lam[m] = rho[m] * A.cvk;
    T0[m] = T;
    const int b = (j0 + m) * FW + i;
    sT[b] = T;
    sUx[b] = ux;
    sUy[b] = uy;
    sLam[b] = lam[m];
  }
  __syncthreads();

  // ---- coefficients (every row of the run; see energy_tile for the form)
  float Dx[R + 2], Sy[R + 2], uyc[R + 2];
#pragma unroll
  for (int m = -1; m <= R; ++m) {
    const int j = min(max(j0 + m, 0), FH - 1);
    Dx[m + 1] = sUx[j * FW + ie] - sUx[j * FW + iw];
    Sy[m + 1] = sUy[j * FW + ie] + sUy[j * FW + iw];
    uyc[m + 1] = sUy[j * FW + i];
  }
  const float lamS_run = sLam[max(j0 - 1, 0) * FW + i];
  const float lamN_run = sLam[min(j0 + R, FH - 1) * FW + i];
  const float two_k = 2.f * A.kd;
  const float Rc = A.R / A.cv, akc = A.a * A.kappa / A.cv;
  float cf[R][NCOEF];
  float rS = 1.f / (lam[0] + lamS_run);  // 1 / (lambda + lambda_S) of the run's first row
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int b = (j0 + m) * FW;
    const float l = lam[m];
    const float lE = sLam[b + ie], lW = sLam[b + iw];
    const float lN = m + 1 < R ? lam[m + 1] : lamN_run;
    const float lS = m > 0 ? lam[m - 1] : lamS_run;
    const float rN = 1.f / (l + lN);
    const float cE = two_k * lE / (l + lE), cW = two_k * lW / (l + lW);
    const float cN = two_k * lN * rN, cS = two_k * lS * rS;
    rS = rN;  // the next row's south face is this row's north face
    const float ux = sUx[b + i], uy = uyc[m + 1];
    const float divu = Dx[m + 1] * (1.f / 3.f) + (Dx[m + 2] + Dx[m]) * (1.f / 12.f) +
                       (uyc[m + 2] - uyc[m]) * (1.f / 3.f) + (Sy[m + 2] - Sy[m]) * (1.f / 12.f);
    const float br = A.b * rho[m];
    cf[m][C_AE] = fmaf(ux, -1.f / 3.f, cE);
    cf[m][C_AW] = fmaf(ux, 1.f / 3.f, cW);
    cf[m][C_AN] = fmaf(uy, -1.f / 3.f, cN);
    cf[m][C_AS] = fmaf(uy, 1.f / 3.f, cS);
    cf[m][C_P] = (ux + uy) * (1.f / 12.f);
    cf[m][C_Q] = (ux - uy) * (1.f / 12.f);
    cf[m][C_AS_T] = divu * Rc / (1.f - br);
    cf[m][C_BS] = divu * akc * rho[m] / fmaf(br, 2.f - br, 1.f);
  }

  // ---- RK4 stages (Eq. 18)
  const float dt = A.dt;
  const float k1 = 1.f + A.kappa;
  float cur[R], acc[R];
  float eh = 0.f, el = 0.f;
#pragma unroll
  for (int m = 0; m < R; ++m) {
    cur[m] = T0[m];
    acc[m] = 0.f;
  }
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    const float* In = k == 1 ? sT : (k == 3 ? sB : sA);
    float* Out = k == 2 ? sB : sA;
    const float cnext = k == 3 ? dt : 0.5f * dt;
    const float wacc = k == 1 ? 1.f : 2.f;
    const int js = max(j0 - 1, 0), jn = min(j0 + R, FH - 1);
    float Es = In[js * FW + ie], Ws = In[js * FW + iw];
    float Ec = In[j0 * FW + ie], Wc = In[j0 * FW + iw];
    float prev = In[js * FW + i];
    const float Cn = In[jn * FW + i];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int ja = m + 1 < R ? j0 + m + 1 : jn;
      const float En = In[ja * FW + ie], Wn = In[ja * FW + iw];
      const float Tp = cur[m];
      const float TS = prev;
      prev = Tp;
      const float TN = m + 1 < R ? cur[m + 1] : Cn;
      const float* c = cf[m];
      float kk = c[C_AE] * (Ec - Tp);
      kk = fmaf(c[C_AW], Wc - Tp, kk);
      kk = fmaf(c[C_AN], TN - Tp, kk);
      kk = fmaf(c[C_AS], TS - Tp, kk);
      kk = fmaf(-c[C_P], En - Ws, kk);
      kk = fmaf(-c[C_Q], Es - Wn, kk);
      const float sTr = sqrtf(fmaxf(Tp, 0.f) * A.invTc);
      kk -= fmaf(c[C_AS_T], Tp, c[C_BS] * sTr * fmaf(-A.kappa, sTr, k1));
      if (k < 4) {
        acc[m] = fmaf(wacc, kk, acc[m]);
        cur[m] = fmaf(cnext, kk, T0[m]);
      } else {
        const int j = j0 + m;
        if (own_col && j >= H && j < H + TY) {
          const float Tnew = T0[m] + dt * (1.f / 6.f) * (acc[m] + kk);
          if (nonfinite(Tnew)) err |= ERR_NONFINITE;
          T_out[(gy0 + m) * nx + gx] = Tnew;
          if (last) ff_add(eh, el, Tnew * (rho[m] * A.cv));
        }
      }
      Es = Ec;
      Ws = Wc;
      Ec = En;
      Wc = Wn;
    }
    if (k < 4) {
#pragma unroll
      for (int m = 0; m < R; ++m) Out[(j0 + m) * FW + i] = cur[m];
      __syncthreads();
    }
  }
  float ah[NEPART] = {0.f, 0.f, 0.f, eh}, al[NEPART] = {0.f, 0.f, 0.f, el};
  if (err) atomicOr(&s_err, err);
  block_partials<NT, NEPART>(ah, al, s_red, A.epart + (long long)part * NEPART, s > 1);
  if (tid == 0 && s_err) atomicOr(&A.state->error_flags, s_err);
}

template <int R, int NPH>
__device__ __forceinline__ void energy_tile(const StepArgs& A, int bx, int by, int part, float* sm, int s, int nsub) {
  constexpr int FW = EN_FW, H = EN_H, FH = R * NPH, TY = FH - 2 * H, FN = FW * FH, NT = FW * NPH;
  static_assert(TY == EN_TY && FH == EN_FH, "energy tile geometry");
  float* const sT = sm;           // T^n on the frame: stage-1 input
  float* const sA = sm + FN;      // stage outputs (stages 1 and 3)
  float* const sB = sm + 2 * FN;  // stage outputs (stage 2); u_x during the coefficient pass
  float* const sUy = sm + 3 * FN;
  float* const sLam = sm + 4 * FN;
  float* const sUx = sB;
  __shared__ float s_red[NT / 32][NEPART][2];
  __shared__ int s_err;

  const float* __restrict__ T_in = s == 1 ? A.T_in : substep_buffer(A, s - 1, nsub);
  float* __restrict__ T_out = substep_buffer(A, s, nsub);
  const bool last = s == nsub;
  const Geo g = make_geo(A);
  const int nx = A.nx, ny = A.ny, W = A.W;
  const int NC = nx * ny;
  const float* __restrict__ rho_n = A.mom;
  const float* __restrict__ ux_n = A.mom + NC;
  const float* __restrict__ uy_n = A.mom + 2 * NC;
  const int x0 = bx * EN_TX, y0 = by * TY;
  const int tid = threadIdx.x;
  const int i = tid & (FW - 1), jp = tid / FW;
  const int j0 = jp * R;                 // first frame row of the run
  const int gy0 = y0 - H + j0;           // its lattice row
  const int gxu = x0 - H + i;
  const int gx = wrapx(gxu, nx);
  const bool own_col = i >= H && i < H + EN_TX && gxu < nx;
  const bool top_open = g.top_open;
  auto wall_lam = [&](int row) -> float { return g.top_wall && row == ny - 1 ? A.lambda_top : A.lambda_w; };
  if (tid == 0) s_err = 0;
  int err = 0;

  // ---- load T (wall values on Dirichlet rows), rho^n, u^n and lambda; frame
  // rows above the lattice hold copies of row ny - 1, rows below it zeros
  float T0[R], rho[R], lam[R];
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int j = j0 + m, gy = gy0 + m;
    float T = 0.f, ux = 0.f, uy = 0.f;
    rho[m] = 0.f;
    lam[m] = A.lambda_w;
    if (gy >= 0) {
      const int gr = gy < ny ? gy : ny - 1;
      const int c = gr * nx + gx;
      T = g.dirichlet_row(gr) ? (gr == 0 ? A.T_bottom : A.T_top) : __ldg(T_in + c);
      if (g.solid_row(gr)) {
        lam[m] = wall_lam(gr);
      } else {
        rho[m] = __ldg(rho_n + c);
        ux = __ldg(ux_n + c);
        uy = __ldg(uy_n + c);
        lam[m] = rho[m] * A.cvk;
      }
    }
    T0[m] = T;
    sT[j * FW + i] = T;
    sUx[j * FW + i] = ux;
    sUy[j * FW + i] = uy;
    sLam[j * FW + i] = lam[m];
  }
  __syncthreads();

  // ---- coefficients on ring 3 (frame rows 1 .. FH-2, every column; the two
  // edge columns read neighbours of the adjacent rows and are never used)
  // div u (Eq. 19), separable: with Dx(r) = u_x(E) - u_x(W) and Sy(r) = u_y(E) + u_y(W)
  // of row r, div u = Dx(0)/3 + (Dx(+1) + Dx(-1))/12 + (u_y(N) - u_y(S))/3 + (Sy(+1) - Sy(-1))/12
  float Dx[R + 2], Sy[R + 2], uyc[R + 2];
#pragma unroll
  for (int m = -1; m <= R; ++m) {
    const int j = min(max(j0 + m, 0), FH - 1);
    const int b = j * FW + i;
    Dx[m + 1] = sUx[b + 1] - sUx[b - 1 < 0 ? 0 : b - 1];
    Sy[m + 1] = sUy[b + 1 < FN ? b + 1 : FN - 1] + sUy[b - 1 < 0 ? 0 : b - 1];
    uyc[m + 1] = sUy[b];
  }
  const float lamS_run = sLam[max(j0 - 1, 0) * FW + i];
  const float lamN_run = sLam[min(j0 + R, FH - 1) * FW + i];
  float cf[R][NCOEF];
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int j = j0 + m, gy = gy0 + m;
#pragma unroll
    for (int q = 0; q < NCOEF; ++q) cf[m][q] = 0.f;
    if (j < 1 || j >= FH - 1 || gy < 0 || gy >= ny) continue;  // warp-uniform
    const bool solid = g.solid_row(gy);
    if (g.dirichlet_row(gy)) continue;  // T held: K = 0
    const int b = j * FW + i;
    const float lE = sLam[b + 1], lW = sLam[b - 1];
    float lN = m + 1 < R ? lam[m + 1] : lamN_run;
    const float lS = m > 0 ? lam[m - 1] : lamS_run;
    if (top_open && gy == ny - 1) lN = lam[m];  // zero-gradient ghost above an open top
    const float ircv = solid ? A.inv_rcv_w : 1.f / (rho[m] * A.cv);
    const float cE = harm(lam[m], lE) * ircv, cW = harm(lam[m], lW) * ircv;
    const float cN = harm(lam[m], lN) * ircv;
    // row 0 under an imposed flux (Section 3.3): no conductive flux through its
    // bottom face (T below is the edge copy); q_in enters instead (added in the stages)
    const float cS = gy == 0 ? 0.f : harm(lam[m], lS) * ircv;
    if (solid) {
      cf[m][C_AE] = cE;
      cf[m][C_AW] = cW;
      cf[m][C_AN] = cN;
      cf[m][C_AS] = cS;
      continue;
    }
    // (above an open top the frame holds copies of row ny - 1: the zero-gradient ghost)
    const float ux = sUx[b], uy = uyc[m + 1];
    const float divu = Dx[m + 1] * (1.f / 3.f) + (Dx[m + 2] + Dx[m]) * (1.f / 12.f) +
                       (uyc[m + 2] - uyc[m]) * (1.f / 3.f) + (Sy[m + 2] - Sy[m]) * (1.f / 12.f);
    const float br = A.b * rho[m];
    const float Ar = rho[m] * A.R / (1.f - br);
    const float Br = A.a * rho[m] * rho[m] * A.kappa / (1.f + 2.f * br - br * br);
    cf[m][C_AE] = cE - ux * (1.f / 3.f);
    cf[m][C_AW] = cW + ux * (1.f / 3.f);
    cf[m][C_AN] = cN - uy * (1.f / 3.f);
    cf[m][C_AS] = cS + uy * (1.f / 3.f);
    cf[m][C_P] = (ux + uy) * (1.f / 12.f);
    cf[m][C_Q] = (ux - uy) * (1.f / 12.f);
    cf[m][C_AS_T] = Ar * ircv * divu;
    cf[m][C_BS] = Br * ircv * divu;
  }

  // ---- RK4 stages (Eq. 18): stage k on ring 4 - k; the run's own values in registers
  const float dt = A.dt;
  const float qc = A.q_in * A.inv_rcv_w;  // row 0 under an imposed flux (solid)
  const float k1 = 1.f + A.kappa;
  float cur[R], acc[R];
  float ah[NEPART], al[NEPART];
#pragma unroll
  for (int q = 0; q < NEPART; ++q) ah[q] = al[q] = 0.f;
#pragma unroll
  for (int m = 0; m < R; ++m) {
    cur[m] = T0[m];
    acc[m] = 0.f;
  }
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    const float* In = k == 1 ? sT : (k == 3 ? sB : sA);
    float* Out = k == 2 ? sB : sA;
    const float cnext = k == 3 ? dt : 0.5f * dt;
    const float wk = (k == 1 || k == 4) ? dt * (1.f / 6.f) : dt * (2.f / 6.f);
    const float wacc = k == 1 ? 1.f : 2.f;
    const int r = 4 - k;
    // neighbours of the run: columns i - 1 and i + 1 as a three-row window
    // rolling up the run, and column i just below and above it
    const int ie = i + 1 < FW ? i + 1 : i, iw = i > 0 ? i - 1 : i;
    const int js = max(j0 - 1, 0), jn = min(j0 + R, FH - 1);
    float Es = In[js * FW + ie], Ws = In[js * FW + iw];
    float Ec = In[j0 * FW + ie], Wc = In[j0 * FW + iw];
    float prev = In[js * FW + i];  // stage input of the row below the current one
    const float Cn = In[jn * FW + i];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int j = j0 + m, gy = gy0 + m;
      const int ja = m + 1 < R ? j + 1 : jn;
      const float En = In[ja * FW + ie], Wn = In[ja * FW + iw];
      const float Tp = cur[m];
      const float TS = prev;
      prev = Tp;
      if (!(j < H - r || j >= H + TY + r || gy < 0 || gy >= ny)) {  // warp-uniform ring test
        float TN = m + 1 < R ? cur[m + 1] : Cn;
        float TNE = En, TNW = Wn;
        if (top_open && gy == ny - 1) {  // zero-gradient ghost above an open top
          TN = Tp;
          TNE = Ec;
          TNW = Wc;
        }
        const float* c = cf[m];
        float kk = c[C_AE] * (Ec - Tp);
        kk = fmaf(c[C_AW], Wc - Tp, kk);
        kk = fmaf(c[C_AN], TN - Tp, kk);
        kk = fmaf(c[C_AS], TS - Tp, kk);
        kk = fmaf(-c[C_P], TNE - Ws, kk);
        kk = fmaf(-c[C_Q], Es - TNW, kk);
        const float sTr = sqrtf(fmaxf(Tp, 0.f) * A.invTc);
        kk -= fmaf(c[C_AS_T], Tp, c[C_BS] * sTr * fmaf(-A.kappa, sTr, k1));
        if (gy == 0 && g.bottom_flux) kk += qc;
        const bool own = own_col && j >= H && j < H + TY;
        if (own && (gy == 1 || gy == W || (g.top_wall && gy == ny - 2))) {
          // RK-weighted conductive fluxes through the wall faces (q_bottom, q_interface, q_top)
          const float lc = sLam[j * FW + i];
          const float lS = harm(lc, sLam[(j - 1) * FW + i]);
          if (gy == 1) ff_add(ah[EP_QB], al[EP_QB], wk * lS * (TS - Tp));
          if (gy == W) ff_add(ah[EP_QI], al[EP_QI], wk * lS * (TS - Tp));
          if (g.top_wall && gy == ny - 2)
            ff_add(ah[EP_QT], al[EP_QT], wk * harm(lc, sLam[(j + 1) * FW + i]) * (Tp - TN));
        }
        if (k < 4) {
          acc[m] = fmaf(wacc, kk, acc[m]);
          cur[m] = fmaf(cnext, kk, T0[m]);
        } else if (own) {
          const float Tnew = T0[m] + dt * (1.f / 6.f) * (acc[m] + kk);
          if (nonfinite(Tnew)) err |= ERR_NONFINITE;
          T_out[gy * nx + gx] = Tnew;
          // sensible energy rho cv T (lambda = rho cv k in the fluid)
          if (last) ff_add(ah[EP_E], al[EP_E], Tnew * (g.solid_row(gy) ? A.rcv_w : sLam[j * FW + i] * A.inv_k));
        }
      }
      Es = Ec;
      Ws = Wc;
      Ec = En;
      Wc = Wn;
    }
    if (k < 4) {
#pragma unroll
      for (int m = 0; m < R; ++m) Out[(j0 + m) * FW + i] = cur[m];
      __syncthreads();
    }
  }
  if (err) atomicOr(&s_err, err);
  // fluxes add up over the sub-steps; the energy of T^{n+1} comes from the last
  block_partials<NT, NEPART>(ah, al, s_red, A.epart + (long long)part * NEPART, s > 1);
  if (tid == 0 && s_err) atomicOr(&A.state->error_flags, s_err);
}

template <int R, int NPH, int MINB>
__global__ void __launch_bounds__(64 * NPH, MINB) k_energy(const StepArgs A, int s, int nsub) {
  extern __shared__ float sm[];
  const int part = blockIdx.y * gridDim.x + blockIdx.x;
  if (energy_interior(A, blockIdx.y * EN_TY))
    energy_tile_int<R, NPH>(A, blockIdx.x, blockIdx.y, part, sm, s, nsub);
  else
    energy_tile<R, NPH>(A, blockIdx.x, blockIdx.y, part, sm, s, nsub);
}

template <int R, int NPH, int MINB>
__global__ void __launch_bounds__(64 * NPH, MINB) k_energy_batch(const StepArgs P, const DomArgs* __restrict__ desc,
                                                                 const int2* __restrict__ blk,
                                                                 const int* __restrict__ active, int s, int nsub) {
  extern __shared__ float sm[];
  __shared__ DomArgs sD;
  __shared__ int s_act;
  __shared__ int2 s_bl;
  __shared__ float2 s_lg;
  if (!batch_prologue<64 * NPH>(desc, blk, active, nullptr, sD, s_bl, s_lg, s_act)) return;
  StepArgs A = P;
  apply_dom(A, sD);
  const int local = s_bl.y;
  const int tx = (A.nx + EN_TX - 1) / EN_TX;
  const int by = local / tx;
  if (energy_interior(A, by * EN_TY))
    energy_tile_int<R, NPH>(A, local % tx, by, local, sm, s, nsub);
  else
    energy_tile<R, NPH>(A, local % tx, by, local, sm, s, nsub);
}

// ------------------------------------------------------------- reduction
// Sums the flow and energy tiles' partials of one domain (one CTA) and updates
// the record: lagged mean density (Eq. 9) and outlet velocity for the next
// step, diagnostics, running sums, flux history.
__device__ __forceinline__ void reduce_split_block(const double* __restrict__ fpart, int nf,
                                                   const double* __restrict__ epart, int ne, DevState* st,
                                                   double inv_nfluid, double inv_nx, double* hist, int hist_cap,
                                                   float2* lag) {
  __shared__ double s_red[8][NFPART + NEPART];
  double v[NFPART + NEPART];
#pragma unroll
  for (int q = 0; q < NFPART + NEPART; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < nf; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NFPART; ++q) v[q] += fpart[(long long)b * NFPART + q];
  }
  for (int b = threadIdx.x; b < ne; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NEPART; ++q) v[NFPART + q] += epart[(long long)b * NEPART + q];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NFPART + NEPART; ++q) {
    const double s = warp_sum(v[q]);
    if (lane == 0) s_red[warp][q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[NFPART + NEPART];
#pragma unroll
    for (int q = 0; q < NFPART + NEPART; ++q) {
      s[q] = 0.0;
      for (int w = 0; w < 8; ++w) s[q] += s_red[w][q];
    }
    st->rho_ave_prev = st->rho_ave;
    st->rho_ave = s[FP_MASS] * inv_nfluid;
    const double ut = s[FP_UTOP] * inv_nx;
    st->u_top = ut;
    st->U = ut > 0.0 ? ut : 0.0;
    st->Uc = st->U / (1.0 + st->U);
    st->step += 1;
    st->mass = s[FP_MASS];
    st->energy = s[NFPART + EP_E];
    st->q_bottom = s[NFPART + EP_QB] * inv_nx;
    st->q_top = s[NFPART + EP_QT] * inv_nx;
    st->q_interface = s[NFPART + EP_QI] * inv_nx;
    st->q_sum += st->q_bottom;
    st->q_count += 1;
    st->vcov = s[FP_VCOV] * inv_nx;
    st->vcov_sum += st->vcov;
    if (hist && st->hist_len < hist_cap) hist[st->hist_len++] = st->q_bottom;
    if (lag) *lag = make_float2((float)st->Uc, (float)st->rho_ave);
  }
}

__global__ void __launch_bounds__(256) k_reduce_split(const double* __restrict__ fpart, int nf,
                                                       const double* __restrict__ epart, int ne, DevState* st,
                                                       double inv_nfluid, double inv_nx, double* hist, int hist_cap) {
  reduce_split_block(fpart, nf, epart, ne, st, inv_nfluid, inv_nx, hist, hist_cap, nullptr);
}

struct SplitReduceArgs {
  const double* fpart;
  const double* epart;
  DevState* state;
  double* hist;
  int nf, ne;
  double inv_nfluid, inv_nx;
};

__global__ void __launch_bounds__(256) k_reduce_split_batch(const SplitReduceArgs* __restrict__ ra,
                                                             const int* __restrict__ active, float2* lag,
                                                             int hist_cap) {
  const int d = blockIdx.x;
  if (!active[d]) return;
  const SplitReduceArgs r = ra[d];
  reduce_split_block(r.fpart, r.nf, r.epart, r.ne, r.state, r.inv_nfluid, r.inv_nx, r.hist, hist_cap, lag + d);
}

}  // namespace hlb
