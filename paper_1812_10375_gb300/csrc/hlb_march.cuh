// Row-marching form of the fused coupled step (Hu & Liu, arXiv 1812.10375).
//
// The same step as step_tile (pull-streaming with bounce-back, Eqs. 1-2;
// rho and psi, Eqs. 5, 7, 28; F = F_m + F_ads + F_b, Eqs. 6, 9, 10; u, Eq. 5;
// MRT collision with Li's forcing, Eqs. 2-4, 8; RK4, Eq. 18, of the energy
// equation, Eq. 17, with harmonic face conductivities, Eqs. 22-26), computed
// by a CTA that owns the full width of a domain (one thread per column, x
// periodic, so no x halo) and a segment [ys, ye) of its rows.  The CTA walks
// up the rows once; at step t of the walk seven phases work on seven rows:
//
//   A   pull row t, rho, psi, T^n                          lag 0, interval 0
//   B   forces, u; collide and store row t-1              lag 1, interval 1
//   C   face conductivities, 1/(rho cv), latent-heat
//       coefficients of row t-2                            lag 2, interval 2
//   S1  RK4 stage 1 of row t-4                             lag 4, interval 0
//   S2  stage 2 of row t-5                                 lag 5, interval 1
//   S3  stage 3 of row t-6                                 lag 6, interval 2
//   S4  stage 4 of row t-8, store T^{n+1}                  lag 8, interval 0
//
// Three CTA barriers split a step into three intervals.  A phase reads the
// rows r-1..r+1 of what another phase produced: in this step if the producer
// runs in an earlier interval (lag one row more), else from the previous step
// (lag two rows more), so phases of one interval never wait on each other.
// One walk covers the ring-6 dependency of the energy update in the y
// direction only: the halo recompute is 5 rows above and below a segment
// instead of a ring around every tile.  Row quantities live in shared-memory
// ring buffers of depth 4 or 8 (at least the producer-to-last-consumer
// distance, without a slot being rewritten in the interval that last reads
// it); the walk is unrolled by 8 so that every ring slot is a compile-time
// constant.  HBM traffic is the algorithmic 36 + 36 B of populations and
// 4 + 4 B of temperature per cell, plus the re-read of 10 halo rows per
// segment, which mostly hits L2.
#pragma once
#include "hlb_kernels.cuh"

namespace hlb {

constexpr int MARCH_MAX_NX = 512;  // one column per thread, at most 512 threads
constexpr int MARCH_DS = 4, MARCH_DL = 8;  // short and long ring depths; the walk is unrolled by MARCH_DL
constexpr int LAG_B = 1, LAG_C = 2, LAG_S1 = 4, LAG_S2 = 5, LAG_S3 = 6, LAG_S4 = 8;
constexpr int MARCH_LAG_MAX = LAG_S4;
// segment heights the host may choose (the autotuner times each)
#define HLB_MARCH_SEGMENTS(X) X(32) X(48) X(64)

// ring quantities of the short and of the long depth
enum { R3_PSI = 0, R3_RHO, R3_T1, R3_T2, R3_T3, NR3 };
enum { R6_TN = 0, R6_UX, R6_UY, R6_LE, R6_LN, R6_IRCV, R6_AS, R6_BS, NR6 };

__host__ __device__ constexpr int march_row_stride(int nx) { return (nx + 31) / 32 * 32; }
// Prefetch ring: the nine pulled populations and T^n of the next two rows to
// pull, copied global -> shared by cp.async while the CTA works on earlier rows.
constexpr int MARCH_PF = 10, MARCH_DP = 2;
// values per column: the rings, the prefetch ring and a pad word so that the stride is odd
__host__ __device__ constexpr int march_nq() {
  return (MARCH_DS * NR3 + MARCH_DL * NR6 + MARCH_DP * MARCH_PF) | 1;
}
constexpr int MARCH_PF_OFF = MARCH_DS * NR3 + MARCH_DL * NR6;
__host__ __device__ constexpr int march_smem_floats(int nx) { return march_nq() * march_row_stride(nx); }

// Ring slot of a row: rows are >= 0 when stored, the phase PH = t mod 8 is a
// template parameter, so (t - lag) mod D is a constant.
template <int PH, int LAG, int D>
struct Slot {
  static constexpr int v = (((PH - LAG) % D) + D) % D;
};

// Shared memory holds the rings column by column: column c's NQ values (an
// odd stride, so 32 consecutive columns fall in 32 different banks) start at
// c * NQ, and quantity q of ring slot s sits at a constant offset within
// them.  A row view adds that constant to the column's base, so every ring
// access compiles to a register base plus an immediate offset.
constexpr int MARCH_NQ = march_nq();

struct SRow {
  float* b;  // sm + (constant offset of the quantity's slot)
  __device__ __forceinline__ float& operator[](int col) const { return b[col * MARCH_NQ]; }
};

struct MarchCtx {
  float* sm;
  __device__ __forceinline__ SRow q3(int q, int slot) const { return SRow{sm + q * MARCH_DS + slot}; }
  __device__ __forceinline__ SRow q6(int q, int slot) const {
    return SRow{sm + MARCH_DS * NR3 + q * MARCH_DL + slot};
  }
};

// Per-thread state that lives across the phases of the walk.
struct MarchThread {
  int i, ie, iw;  // column, east and west neighbour columns (periodic)
  int xm, xp;     // same, in lattice x
  bool act;       // i < nx
  float gw;       // wetting strength of the column (Eq. 10)
  float* pf;      // this column's prefetch ring in shared memory
  float f0[9];    // pulled populations of row t (A) ...
  float f1[9];    // ... and of row t - 1 (B collides them)
  float rho0;     // rho of row t (A) ...
  float rho1;     // ... and of row t - 1 (B)
  float ac[5];    // RK accumulators K1 + 2 K2 + 2 K3 of rows t-4 .. t-8
  float tn[5];    // T^n of rows t-4 .. t-8
  // partial sums of the segment: mass and energy compensated (hi, lo); the
  // wall-row quantities get at most four terms per thread, kept in plain FP32
  float mh, ml, eh, el;
  float vcov, utop, qb, qt, qi;
  int err;
};

// Row classes (uniform over the CTA).
struct MarchRows {
  int nx, ny, W, ys, ye, t_first;
  bool top_wall, top_open, bottom_flux;
  __device__ __forceinline__ bool solid(int y) const { return y < W || (top_wall && y == ny - 1); }
  __device__ __forceinline__ bool dirichlet(int y) const {
    return (y == 0 && !bottom_flux) || (top_wall && y == ny - 1);
  }
  // rows a phase covers: [ys - lo, ye + hi) within the lattice; row ny is
  // the zero-gradient ghost above an open top, copied from row ny - 1 by
  // every phase whose range reaches the top row
  __device__ __forceinline__ bool in(int y, int lo, int hi) const {
    return y >= ys - lo && y < ye + hi && y >= 0 && y < ny;
  }
  __device__ __forceinline__ bool ghost(int y, int lo, int hi) const { return top_open && y == ny && in(y - 1, lo, hi); }
};

// all but the most recent group complete: the row pulled now has arrived, the next one may be in flight
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Issue the pull of row y (the sources of pull(): pull-streaming, halfway
// bounce-back next to solid rows, open-top rules) and of T^n(y) as cp.async
// copies into prefetch slot y mod 2 of this column.  Values that are not
// copies (the constant-density top row, Dirichlet temperatures) are stored
// directly; the convective outlet's raw sources are copied and combined with
// the outlet memory when the row is used (march_A).
__device__ __forceinline__ void march_fetch(const StepArgs& A, const MarchRows& R, MarchThread& th, int y) {
  if (!th.act || y < 0 || y >= R.ny) return;
  float* d = th.pf + (y & 1) * MARCH_PF;
  const int nx = R.nx, x = th.i;
  const int r0 = y * nx;
  if (R.dirichlet(y))
    d[9] = y == 0 ? A.T_bottom : A.T_top;
  else
    cp_async4(d + 9, A.T_in + r0 + x);
  if (R.solid(y)) return;
  const int P = (int)A.plane;
  const float* __restrict__ F = A.f_in;
  const bool bb_s = R.solid(y - 1);
  const bool sol_n = R.solid(y + 1 < R.ny ? y + 1 : R.ny - 1);
  const bool open_n = R.top_open && y == R.ny - 1;
  const int rs = r0 - nx, rn = r0 + nx, xm = th.xm, xp = th.xp;
  cp_async4(d + 0, F + r0 + x);
  cp_async4(d + 1, F + 1 * P + r0 + xm);
  cp_async4(d + 3, F + 3 * P + r0 + xp);
  if (bb_s) {
    cp_async4(d + 2, F + 4 * P + r0 + x);
    cp_async4(d + 5, F + 7 * P + r0 + x);
    cp_async4(d + 6, F + 8 * P + r0 + x);
  } else {
    cp_async4(d + 2, F + 2 * P + rs + x);
    cp_async4(d + 5, F + 5 * P + rs + xm);
    cp_async4(d + 6, F + 6 * P + rs + xp);
  }
  if (open_n) {
    if (A.top_bc == TOP_CONST_RHO) {
      const float dr = A.rho_v - A.rho_ref;
      d[4] = dr * (1.f / 9.f);
      d[7] = dr * (1.f / 36.f);
      d[8] = dr * (1.f / 36.f);
    } else {
      cp_async4(d + 4, F + 4 * P + r0 + x);
      cp_async4(d + 7, F + 7 * P + r0 + xp);
      cp_async4(d + 8, F + 8 * P + r0 + xm);
    }
  } else if (sol_n) {
    cp_async4(d + 4, F + 2 * P + r0 + x);
    cp_async4(d + 7, F + 5 * P + r0 + x);
    cp_async4(d + 8, F + 6 * P + r0 + x);
  } else {
    cp_async4(d + 4, F + 4 * P + rn + x);
    cp_async4(d + 7, F + 7 * P + rn + xp);
    cp_async4(d + 8, F + 8 * P + rn + xm);
  }
}

// Phase A: row y = t.  rho, psi and T^n of the row into the rings; the pulled
// populations stay in registers for the collision of the next iteration.
template <int PH>
__device__ __forceinline__ void march_A(const StepArgs& A, const MarchRows& R, const MarchCtx& C, MarchThread& th,
                                        int y, float Uc) {
  constexpr int s3 = Slot<PH, 0, MARCH_DS>::v, s6 = Slot<PH, 0, MARCH_DL>::v;
  const SRow psi = C.q3(R3_PSI, s3);
  const SRow rho = C.q3(R3_RHO, s3);
  const SRow tn = C.q6(R6_TN, s6);
  if (R.in(y, 5, 5)) {
    cp_async_wait_prev();
    const float* d = th.pf + (y & 1) * MARCH_PF;
    const float T = d[9];
    if (th.act) {
      if (!R.solid(y)) {
#pragma unroll
        for (int q = 0; q < 9; ++q) th.f0[q] = d[q];
        if (A.top_bc == TOP_CONVECTIVE && y == R.ny - 1) {
          // f_i(top) = [f_i^{n-1}(top) + U f_i^n(top-1)] / (1 + U) as prev + Uc (below - prev),
          // Uc = U / (1 + U) from FP64 (pull() evaluates the same expression)
          const float p4 = A.ftop_in[th.i], p7 = A.ftop_in[R.nx + th.i], p8 = A.ftop_in[2 * R.nx + th.i];
          th.f0[4] = p4 + Uc * (th.f0[4] - p4);
          th.f0[7] = p7 + Uc * (th.f0[7] - p7);
          th.f0[8] = p8 + Uc * (th.f0[8] - p8);
        }
      }
      tn[th.i] = T;
      if (R.solid(y)) {
        psi[th.i] = 0.f;
        rho[th.i] = 0.f;
      } else {
        const float r = A.rho_ref + sum9(th.f0);
        float p2 = pr_psi2(A, r, A.eos_T_fixed ? A.Ts : T);
        if (!(p2 >= 0.f)) {
          th.err |= ERR_PSI_NEG;
          p2 = 0.f;
        }
        psi[th.i] = sqrtf(p2);
        rho[th.i] = r;
        th.rho0 = r;
      }
    }
  } else if (R.ghost(y, 5, 5)) {
    constexpr int p3 = Slot<PH, 1, MARCH_DS>::v, p6 = Slot<PH, 1, MARCH_DL>::v;
    if (th.act) {
      psi[th.i] = C.q3(R3_PSI, p3)[th.i];
      rho[th.i] = C.q3(R3_RHO, p3)[th.i];
      tn[th.i] = C.q6(R6_TN, p6)[th.i];
    }
  }
}

// Phase B: row y = t - 1.  F (Eqs. 6, 9, 10) and u (Eq. 5) for rows within 4
// of the segment; the collision (Eqs. 2-4, 8) and the store of f* for the
// segment's own rows.
template <int PH>
__device__ __forceinline__ void march_B(const StepArgs& A, const MarchRows& R, const MarchCtx& C, MarchThread& th,
                                        int y, float rho_ave) {
  constexpr int s3 = Slot<PH, 1, MARCH_DS>::v, s3n = Slot<PH, 0, MARCH_DS>::v, s3s = Slot<PH, 2, MARCH_DS>::v;
  constexpr int s6 = Slot<PH, 1, MARCH_DL>::v;
  const SRow ux_r = C.q6(R6_UX, s6);
  const SRow uy_r = C.q6(R6_UY, s6);
  if (R.in(y, 4, 4)) {
    if (!th.act) return;
    const int i = th.i;
    if (R.solid(y)) {
      ux_r[i] = 0.f;
      uy_r[i] = 0.f;
      return;
    }
    const SRow P = C.q3(R3_PSI, s3);
    const SRow PN = C.q3(R3_PSI, s3n);
    const SRow PS = C.q3(R3_PSI, s3s);
    const float psi = P[i], rho = th.rho1;
    const bool sol_s = R.solid(y - 1);
    const bool sol_n = R.solid(y + 1 < R.ny ? y + 1 : R.ny - 1);
    // Eq. (6); a solid neighbour carries psi(x)
    const float pE = P[th.ie], pW = P[th.iw];
    const float pN = sol_n ? psi : PN[i];
    const float pS = sol_s ? psi : PS[i];
    const float pNE = sol_n ? psi : PN[th.ie];
    const float pNW = sol_n ? psi : PN[th.iw];
    const float pSE = sol_s ? psi : PS[th.ie];
    const float pSW = sol_s ? psi : PS[th.iw];
    const float sx = (pE - pW) * (1.f / 3.f) + ((pNE - pNW) + (pSE - pSW)) * (1.f / 12.f);
    const float sy = (pN - pS) * (1.f / 3.f) + ((pNE + pNW) - (pSE + pSW)) * (1.f / 12.f);
    const float Fmx = -A.G * psi * sx;
    const float Fmy = -A.G * psi * sy;
    // Eq. (10) with weights omega/3: solid rows are whole rows, so only the
    // normal component (1/9 + 2/36) (s_N - s_S) remains
    const float Fay = th.gw * psi * psi * ((float)sol_n - (float)sol_s) * (1.f / 6.f);
    const float Fx = Fmx;
    const float Fy = Fmy + Fay + (rho - rho_ave) * A.g_y;  // Eq. (9)
    const float* f = th.f1;
    const float jx = (f[1] - f[3]) + ((f[5] - f[6]) - (f[7] - f[8]));
    const float jy = (f[2] - f[4]) + ((f[5] + f[6]) - (f[7] + f[8]));
    const float irho = 1.f / rho;
    const float ux = (jx + 0.5f * Fx) * irho;
    const float uy = (jy + 0.5f * Fy) * irho;
    ux_r[i] = ux;
    uy_r[i] = uy;
    if (y >= R.ys && y < R.ye) {
      const float fsum = collide_store(A, f, rho, ux, uy, Fx, Fy, A.G * A.G * (sx * sx + sy * sy), y * R.nx + i);
      if (nonfinite(fsum)) th.err |= ERR_NONFINITE;
      ff_add(th.mh, th.ml, rho);
      if (y == A.W && rho < A.rho_mid) th.vcov += 1.f;
      if (y == R.ny - 2) th.utop += uy;
      if (A.top_bc == TOP_CONVECTIVE && y == R.ny - 1) {
        A.ftop_out[i] = f[4];
        A.ftop_out[R.nx + i] = f[7];
        A.ftop_out[2 * R.nx + i] = f[8];
      }
    }
  } else if (R.ghost(y, 4, 4)) {
    constexpr int p6 = Slot<PH, 2, MARCH_DL>::v;
    if (th.act) {
      ux_r[th.i] = C.q6(R6_UX, p6)[th.i];
      uy_r[th.i] = C.q6(R6_UY, p6)[th.i];
    }
  }
}

// Phase C: row y = t - 2.  Face conductivities (Eq. 25) for rows [ys - 4,
// ye + 3) (stage 1 on row ys - 3 needs the north face of row ys - 4), and
// 1/(rho cv) and the latent-heat coefficients for rows [ys - 3, ye + 3); lambda =
// rho cv k in the fluid (Section 2.2), lambda_w in solid rows.
template <int PH>
__device__ __forceinline__ void march_C(const StepArgs& A, const MarchRows& R, const MarchCtx& C,
                                        const MarchThread& th, int y) {
  constexpr int s3 = Slot<PH, 2, MARCH_DS>::v, s3n = Slot<PH, 1, MARCH_DS>::v;
  constexpr int s6 = Slot<PH, 2, MARCH_DL>::v, s6n = Slot<PH, 1, MARCH_DL>::v, s6s = Slot<PH, 3, MARCH_DL>::v;
  if (!R.in(y, 4, 3) || !th.act) return;
  const int i = th.i;
  const float cvk = A.cvk;
  // conductivity of a solid row: the heater's, or the top wall's (Section 3.2)
  auto wall_lam = [&](int row) -> float { return R.top_wall && row == R.ny - 1 ? A.lambda_top : A.lambda_w; };
  const SRow RH = C.q3(R3_RHO, s3);
  const bool solid = R.solid(y);
  const float lam = solid ? wall_lam(y) : RH[i] * cvk;
  {
    const float le = solid ? wall_lam(y) : RH[th.ie] * cvk;
    C.q6(R6_LE, s6)[i] = 2.f * lam * le / (lam + le);
  }
  {
    const int yn = y + 1 < R.ny ? y + 1 : R.ny - 1;
    const float ln = R.solid(yn) ? wall_lam(yn) : C.q3(R3_RHO, s3n)[i] * cvk;
    C.q6(R6_LN, s6)[i] = 2.f * lam * ln / (lam + ln);
  }
  if (y < R.ys - 3) return;  // the fourth halo row only needs its north face
  const SRow ircv_r = C.q6(R6_IRCV, s6);
  const SRow as_r = C.q6(R6_AS, s6);
  const SRow bs_r = C.q6(R6_BS, s6);
  if (solid) {
    ircv_r[i] = A.inv_rcv_w;
    as_r[i] = 0.f;
    bs_r[i] = 0.f;
    return;
  }
  const float rho = RH[i];
  const float ircv = 1.f / (rho * A.cv);
  const SRow UX = C.q6(R6_UX, s6);
  const SRow UXn = C.q6(R6_UX, s6n);
  const SRow UXs = C.q6(R6_UX, s6s);
  const SRow UYn = C.q6(R6_UY, s6n);
  const SRow UYs = C.q6(R6_UY, s6s);
  // div u with the isotropic gradient of Eq. (19)
  const float dux = (UX[th.ie] - UX[th.iw]) * (1.f / 3.f) +
                    ((UXn[th.ie] - UXs[th.iw]) + (UXs[th.ie] - UXn[th.iw])) * (1.f / 12.f);
  const float duy = (UYn[i] - UYs[i]) * (1.f / 3.f) +
                    ((UYn[th.ie] - UYs[th.iw]) + (UYn[th.iw] - UYs[th.ie])) * (1.f / 12.f);
  const float divu = dux + duy;
  const float br = A.b * rho;
  // T (dp/dT)_rho = As' T + Bs' (1 + kappa (1 - sqrt Tr)) sqrt Tr (Eq. 28)
  const float Ar = rho * A.R / (1.f - br);
  const float Br = A.a * rho * rho * A.kappa / (1.f + 2.f * br - br * br);
  ircv_r[i] = ircv;
  as_r[i] = Ar * ircv * divu;
  bs_r[i] = Br * ircv * divu;
}

// Stage K of RK4 (Eq. 18) on row y = t - lag: K(T) of Eq. (17) with the
// face fluxes of Eqs. (22)-(26), the isotropic gradient of Eq. (19) and the
// latent-heat source; stage inputs T_k = T^n + c_k dt K_{k-1}.
template <int PH, int K>
__device__ __forceinline__ void march_S(const StepArgs& A, const MarchRows& R, const MarchCtx& C, MarchThread& th,
                                        int y) {
  constexpr int L = K == 1 ? LAG_S1 : (K == 2 ? LAG_S2 : (K == 3 ? LAG_S3 : LAG_S4));
  constexpr int H = 4 - K;                                // rows within H of the segment
  constexpr int CH = L - LAG_S1;                          // chain index of row t - L
  constexpr int CP = K == 1 ? 0 : (K == 2 ? LAG_S2 - LAG_S1 : LAG_S3 - LAG_S1);  // chain index the stage adds to
  constexpr int c3 = Slot<PH, L, MARCH_DS>::v, c3n = Slot<PH, L - 1, MARCH_DS>::v, c3s = Slot<PH, L + 1, MARCH_DS>::v;
  constexpr int c6 = Slot<PH, L, MARCH_DL>::v, c6n = Slot<PH, L - 1, MARCH_DL>::v, c6s = Slot<PH, L + 1, MARCH_DL>::v;
  // stage input ring: T^n (long ring) for K = 1, T_{K-1} (short ring) otherwise
  SRow Tc, Tcn, Tcs;
  if (K == 1) {
    Tc = C.q6(R6_TN, c6);
    Tcn = C.q6(R6_TN, c6n);
    Tcs = C.q6(R6_TN, c6s);
  } else {
    const int q = K == 2 ? R3_T1 : (K == 3 ? R3_T2 : R3_T3);
    Tc = C.q3(q, c3);
    Tcn = C.q3(q, c3n);
    Tcs = C.q3(q, c3s);
  }
  constexpr int qo = K == 1 ? R3_T1 : (K == 2 ? R3_T2 : R3_T3);
  if (R.in(y, H, H)) {
    if (!th.act) return;
    const int i = th.i;
    const float dt = A.dt;
    const float Tp = Tc[i];
    if (K == 1) th.tn[0] = Tp;
    const float T0 = th.tn[CH];
    float hk = 0.f;
    if (!R.dirichlet(y)) {
      const SRow LE = C.q6(R6_LE, c6);
      const SRow LN = C.q6(R6_LN, c6);
      const SRow LNs = C.q6(R6_LN, c6s);
      const float TE = Tc[th.ie], TW = Tc[th.iw], TN = Tcn[i], TS = Tcs[i];
      // row 0 under an imposed flux (Section 3.3): q_in enters through its bottom face
      const bool bot = y == 0;
      float kk;
      if (bot)
        kk = LE[i] * (TE - Tp) + LE[th.iw] * (TW - Tp) + LN[i] * (TN - Tp) + A.q_in;
      else
        kk = LE[i] * (TE - Tp) + LE[th.iw] * (TW - Tp) + LN[i] * (TN - Tp) + LNs[i] * (TS - Tp);
      kk *= C.q6(R6_IRCV, c6)[i];
      if (!R.solid(y)) {
        const float TNE = Tcn[th.ie], TNW = Tcn[th.iw];
        const float TSE = Tcs[th.ie], TSW = Tcs[th.iw];
        const float gxT = (TE - TW) * (1.f / 3.f) + ((TNE - TSW) + (TSE - TNW)) * (1.f / 12.f);
        const float gyT = (TN - TS) * (1.f / 3.f) + ((TNE - TSW) + (TNW - TSE)) * (1.f / 12.f);
        kk -= C.q6(R6_UX, c6)[i] * gxT + C.q6(R6_UY, c6)[i] * gyT;
        const float sTr = sqrtf(fmaxf(Tp, 0.f) * A.invTc);
        kk -= C.q6(R6_AS, c6)[i] * Tp + C.q6(R6_BS, c6)[i] * (1.f + A.kappa * (1.f - sTr)) * sTr;
      }
      hk = kk;
    }
    if (K == 1) th.ac[0] = 1.f * hk;
    if (K == 2 || K == 3) th.ac[CP] += 2.f * hk;
    if (y >= R.ys && y < R.ye) {
      const float wk = (K == 1 || K == 4) ? dt * (1.f / 6.f) : dt * (2.f / 6.f);
      if (y == 1) th.qb += wk * C.q6(R6_LN, c6s)[i] * (Tcs[i] - Tp);
      if (R.top_wall && y == R.ny - 2) th.qt += wk * C.q6(R6_LN, c6)[i] * (Tp - Tcn[i]);
      if (y == A.W) th.qi += wk * C.q6(R6_LN, c6s)[i] * (Tcs[i] - Tp);
      if (K == 4) {
        const float Tnew = T0 + dt * (1.f / 6.f) * (th.ac[CH] + hk);
        if (nonfinite(Tnew)) th.err |= ERR_NONFINITE;
        A.T_out[y * R.nx + i] = Tnew;
        ff_add(th.eh, th.el, Tnew / C.q6(R6_IRCV, c6)[i]);
      }
    }
    if (K < 4) {
      const float cnext = K == 3 ? dt : 0.5f * dt;
      C.q3(qo, c3)[i] = T0 + cnext * hk;
    }
  } else if (K < 4 && R.ghost(y, H, H)) {
    constexpr int p3 = Slot<PH, L + 1, MARCH_DS>::v;
    if (th.act) C.q3(qo, c3)[th.i] = C.q3(qo, p3)[th.i];
  }
}

// One step of the walk: the seven phases at pipeline position t (t mod 8 =
// PH) in three barrier intervals.
template <int PH>
__device__ __forceinline__ void march_iter(const StepArgs& A, const MarchRows& R, const Geo& g, const MarchCtx& C,
                                           MarchThread& th, int t, float Uc, float rho_ave) {
  march_A<PH>(A, R, C, th, t, Uc);
  march_S<PH, 1>(A, R, C, th, t - LAG_S1);
  march_S<PH, 4>(A, R, C, th, t - LAG_S4);
  __syncthreads();
  march_B<PH>(A, R, C, th, t - LAG_B, rho_ave);
  // prefetch the row after next into the slot phase A has just consumed
  if (t >= R.t_first && R.in(t + 2, 5, 5)) march_fetch(A, R, th, t + 2);
  cp_async_commit();
  march_S<PH, 2>(A, R, C, th, t - LAG_S2);
  __syncthreads();
  march_C<PH>(A, R, C, th, t - LAG_C);
  march_S<PH, 3>(A, R, C, th, t - LAG_S3);
  // rotate the per-row registers: row t becomes t - 1, and so on
#pragma unroll
  for (int q = 0; q < 9; ++q) th.f1[q] = th.f0[q];
  th.rho1 = th.rho0;
#pragma unroll
  for (int q = 4; q > 0; --q) {
    th.ac[q] = th.ac[q - 1];
    th.tn[q] = th.tn[q - 1];
  }
  __syncthreads();
}

// The walk of one segment [ys, ye) of a domain; writes f*^n and T^{n+1} of
// the segment's rows and the segment's partial sums into A.partials[part].
__device__ __forceinline__ void march_segment(const StepArgs& A, int ys, int ye, int part, float* sm, float Uc,
                                              float rho_ave) {
  __shared__ int s_err;
  __shared__ float s_red[MARCH_MAX_NX / 32][NPART][2];
  const Geo g = make_geo(A);
  MarchRows R;
  R.nx = A.nx;
  R.ny = A.ny;
  R.W = A.W;
  R.ys = ys;
  R.ye = ye;
  R.top_wall = g.top_wall;
  R.top_open = g.top_open;
  R.bottom_flux = g.bottom_flux;
  MarchCtx C;
  C.sm = sm;

  MarchThread th;
  th.i = threadIdx.x;
  th.act = th.i < A.nx;
  const int i = th.act ? th.i : 0;
  th.ie = i == A.nx - 1 ? 0 : i + 1;
  th.iw = i == 0 ? A.nx - 1 : i - 1;
  th.xm = th.iw;
  th.xp = th.ie;
  th.gw = th.act ? __ldg(A.Gw + i) : 0.f;
  th.err = 0;
  th.rho0 = th.rho1 = 1.f;
#pragma unroll
  for (int q = 0; q < 9; ++q) th.f0[q] = th.f1[q] = 0.f;
  th.pf = sm + (size_t)th.i * MARCH_NQ + MARCH_PF_OFF;
#pragma unroll
  for (int q = 0; q < 5; ++q) th.ac[q] = th.tn[q] = 0.f;
  th.mh = th.ml = th.eh = th.el = 0.f;
  th.vcov = th.utop = th.qb = th.qt = th.qi = 0.f;
  if (threadIdx.x == 0) s_err = 0;

  // first row of phase A, and the last row of phase S4; the walk starts at a
  // multiple of 8 so that t mod 8 is the unrolled copy's template phase
  const int t_first = ys - 5 > 0 ? ys - 5 : 0;
  const int t_last = ye - 1 + MARCH_LAG_MAX;
  const int t0 = t_first - (t_first % MARCH_DL);
  R.t_first = t_first;
  if (R.in(t_first, 5, 5)) march_fetch(A, R, th, t_first);
  cp_async_commit();
  if (R.in(t_first + 1, 5, 5)) march_fetch(A, R, th, t_first + 1);
  cp_async_commit();
#pragma unroll 1
  for (int t = t0; t <= t_last; t += MARCH_DL) {
    march_iter<0>(A, R, g, C, th, t, Uc, rho_ave);
    march_iter<1>(A, R, g, C, th, t + 1, Uc, rho_ave);
    march_iter<2>(A, R, g, C, th, t + 2, Uc, rho_ave);
    march_iter<3>(A, R, g, C, th, t + 3, Uc, rho_ave);
    march_iter<4>(A, R, g, C, th, t + 4, Uc, rho_ave);
    march_iter<5>(A, R, g, C, th, t + 5, Uc, rho_ave);
    march_iter<6>(A, R, g, C, th, t + 6, Uc, rho_ave);
    march_iter<7>(A, R, g, C, th, t + 7, Uc, rho_ave);
  }

  // per-CTA partials: compensated FP32 through warp and block, FP64 at the end
  float ah[NPART], al[NPART];
  ah[P_MASS] = th.mh;
  al[P_MASS] = th.ml;
  ah[P_ENERGY] = th.eh;
  al[P_ENERGY] = th.el;
  ah[P_QB] = th.qb;
  ah[P_QT] = th.qt;
  ah[P_QI] = th.qi;
  ah[P_UTOP] = th.utop;
  ah[P_VCOV] = th.vcov;
  al[P_QB] = al[P_QT] = al[P_QI] = al[P_UTOP] = al[P_VCOV] = 0.f;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NPART; ++q) {
    if (__any_sync(0xffffffffu, ah[q] != 0.f || al[q] != 0.f)) ff_warp_sum(ah[q], al[q]);
    if (lane == 0) {
      s_red[warp][q][0] = ah[q];
      s_red[warp][q][1] = al[q];
    }
  }
  if (th.err) atomicOr(&s_err, th.err);
  __syncthreads();
  if (threadIdx.x < NPART) {
    const int nw = (blockDim.x + 31) >> 5;
    float hi = s_red[0][threadIdx.x][0], lo = s_red[0][threadIdx.x][1];
    for (int w = 1; w < nw; ++w) ff_merge(hi, lo, s_red[w][threadIdx.x][0], s_red[w][threadIdx.x][1]);
    A.partials[(long long)part * NPART + threadIdx.x] = (double)hi + (double)lo;
  }
  if (threadIdx.x == 0 && s_err) atomicOr(&A.state->error_flags, s_err);
}

// Single domain: block b walks rows [b S, min((b + 1) S, ny)).
__global__ void __launch_bounds__(MARCH_MAX_NX, 1) k_march(const StepArgs A, int S) {
  extern __shared__ float sm[];
  const int ys = blockIdx.x * S;
  const int ye = ys + S < A.ny ? ys + S : A.ny;
  march_segment(A, ys, ye, blockIdx.x, sm, (float)A.state->Uc, (float)A.state->rho_ave);
}

// Batch: block b walks segment blk[b].y of domain blk[b].x (all domains of
// one launch have the same row stride, so the block size and the shared
// memory fit every block of the launch).
__global__ void __launch_bounds__(MARCH_MAX_NX, 1) k_march_batch(const StepArgs P, const DomArgs* __restrict__ desc,
                                                                 const int2* __restrict__ blk,
                                                                 const int* __restrict__ active,
                                                                 const float2* __restrict__ lag, int S) {
  extern __shared__ float sm[];
  __shared__ DomArgs sD;
  __shared__ int s_act;
  __shared__ int2 s_bl;
  __shared__ float2 s_lg;
  {
    const int2 bl = blk[blockIdx.x];
    const int* src = reinterpret_cast<const int*>(desc + bl.x);
    int* dst = reinterpret_cast<int*>(&sD);
    for (int q = threadIdx.x; q < (int)(sizeof(DomArgs) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
    if (threadIdx.x == 0) {
      s_bl = bl;
      s_act = active[bl.x];
      s_lg = lag[bl.x];
    }
  }
  __syncthreads();
  if (!s_act) return;
  StepArgs A = P;
  A.nx = sD.nx;
  A.ny = sD.ny;
  A.W = sD.W;
  A.top_bc = sD.top_bc;
  A.eos_T_fixed = sD.eos_T_fixed;
  A.plane = sD.plane;
  A.T_bottom = sD.T_bottom;
  A.T_top = sD.T_top;
  A.f_in = sD.f_in;
  A.f_out = sD.f_out;
  A.T_in = sD.T_in;
  A.T_out = sD.T_out;
  A.Gw = sD.Gw;
  A.ftop_in = sD.ftop_in;
  A.ftop_out = sD.ftop_out;
  A.partials = sD.partials;
  A.state = sD.state;
  const int ys = s_bl.y * S;
  const int ye = ys + S < A.ny ? ys + S : A.ny;
  march_segment(A, ys, ye, s_bl.y, sm, s_lg.x, s_lg.y);
}

}  // namespace hlb
