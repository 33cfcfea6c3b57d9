// Energy sub-step of the split step in row-walking form (Hu & Liu, arXiv
// 1812.10375, Eqs. 17-19, 22-27): one RK4 sub-step (Eq. 18, dt = 1/N) of the
// energy equation with finite-volume harmonic face conductivities, on rho^n and
// u^n held over the sub-steps.
//
// A CTA of 64 threads owns a strip of 56 output columns of one domain (one
// thread per frame column, a 4-column halo on either side recomputed by the
// neighbouring strips) and a segment of L output rows, and walks up the rows
// once.  At walk step t (row r = t) it loads row r, computes the coefficients
// of Eq. (17) and RK4 stage 1 at row r - 1, stage 2 at row r - 2, stage 3 at
// r - 3 and stage 4 (the new temperature) at r - 4.  A stage at row y reads the
// previous stage at rows y - 1 .. y + 1; the row y + 1 value was produced
// earlier in the same walk step, so four CTA barriers separate the phases.
// Row quantities that neighbouring threads read (T^n, the stage values, u and
// lambda) pass through shared-memory rings of a few rows; everything a thread
// needs only for its own column (the coefficients of the four rows in flight,
// the RK accumulators, T^n, the stage values) stays in registers, addressed by
// row mod 4 with the walk unrolled by four.  The y halo is 4 rows below and 4
// above a segment; every row test depends only on the walk step, so branches
// are uniform across the CTA.
#pragma once
#include "hlb_split.cuh"

namespace hlb {

constexpr int EW_W = 64;      // frame columns = threads per CTA
constexpr int EW_OUT = 56;    // output columns of a strip
constexpr int EW_H = 4;       // x halo
constexpr int EW_RTN = 8;     // depth of the T^n ring
constexpr int EW_R = 4;       // depth of the other rings
constexpr int EW_RPF = 8;     // slots of the prefetch ring (rows r .. r + PF, PF < 8)
// shared floats: T^n ring, three stage rings, u_x, u_y, lambda rings, and the
// prefetch ring (T^n, rho^n, u_x, u_y of the rows the asynchronous copies fill)
constexpr int EW_SMEM_FLOATS = (EW_RTN + 6 * EW_R + 4 * EW_RPF) * EW_W;
constexpr int EW_OFF_TN = 0, EW_OFF_T1 = EW_RTN * EW_W, EW_OFF_T2 = EW_OFF_T1 + EW_R * EW_W,
              EW_OFF_T3 = EW_OFF_T2 + EW_R * EW_W, EW_OFF_UX = EW_OFF_T3 + EW_R * EW_W,
              EW_OFF_UY = EW_OFF_UX + EW_R * EW_W, EW_OFF_LAM = EW_OFF_UY + EW_R * EW_W,
              EW_OFF_PF = EW_OFF_LAM + EW_R * EW_W;
// The rings of the walking kernels, at a fixed layout so that every access is
// an immediate offset from one shared-memory base.
__shared__ __align__(16) float s_walk[EW_SMEM_FLOATS];

// Per-thread state of the walk.  Arrays indexed [row & 3] are row rings; the
// walk is unrolled by four so that every index is a compile-time constant.
struct WalkState {
  float tn[4];      // T^n of rows r .. r-3
  float t1[4], t2[4], t3[4];  // stage values of the rows in flight
  float acc[4];     // K1 + 2 K2 + 2 K3
  float cf[4][NCOEF];
  float rcv[4];     // rho cv of a row (energy sum)
  float qf[4];      // unscaled wall-face conductivity of a wall-flux row
  float dx[4], sy[4], uy[4], lam[4];
  float rho1;       // rho of row r - 1 (coefficient pass)
  float pT, pR, pUx, pUy;  // prefetched row
  float eh, el, qbh, qbl, qih, qil, qth, qtl;
  int err;
};

struct WalkCtx {
  const float* T_in;
  float* T_out;
  const float* rho_n;
  const float* ux_n;
  const float* uy_n;
  int i, ie, iw, gx;
  bool own_col;
  int ys, ye;  // output rows of the segment
  bool last;
  // prefetch in 16-byte pieces (nx a multiple of 4): this thread's piece of
  // row y starts at vsrc + y * nx in the lattice
  const float* vsrc;
};

// RK4 right-hand side at one cell from the coefficient row and the 3 x 3 stencil.
__device__ __forceinline__ float walk_K(const StepArgs& A, const float* c, float Tp, float TE, float TW, float TN,
                                        float TS, float TNE, float TNW, float TSE, float TSW) {
  float kk = c[C_AE] * (TE - Tp);
  kk = fmaf(c[C_AW], TW - Tp, kk);
  kk = fmaf(c[C_AN], TN - Tp, kk);
  kk = fmaf(c[C_AS], TS - Tp, kk);
  kk = fmaf(-c[C_P], TNE - TSW, kk);
  kk = fmaf(-c[C_Q], TSE - TNW, kk);
  const float sTr = sqrtf(fmaxf(Tp, 0.f) * A.invTc);
  return kk - fmaf(c[C_AS_T], Tp, c[C_BS] * sTr * fmaf(-A.kappa, sTr, 1.f + A.kappa));
}

template <bool STEADY>
__device__ __forceinline__ void walk_load(const StepArgs& A, const WalkCtx& C, WalkState& S, int row) {
  if (STEADY) {  // an interior fluid row
    const int c = row * A.nx + C.gx;
    S.pT = __ldg(C.T_in + c);
    S.pR = __ldg(C.rho_n + c);
    S.pUx = __ldg(C.ux_n + c);
    S.pUy = __ldg(C.uy_n + c);
    return;
  }
  S.pT = S.pR = S.pUx = S.pUy = 0.f;
  if (row < 0) return;
  const Geo g = make_geo(A);
  const int gr = row < A.ny ? row : A.ny - 1;  // zero-gradient ghost above the lattice
  const int c = gr * A.nx + C.gx;
  S.pT = g.dirichlet_row(gr) ? (gr == 0 ? A.T_bottom : A.T_top) : __ldg(C.T_in + c);
  if (!g.solid_row(gr)) {
    S.pR = __ldg(C.rho_n + c);
    S.pUx = __ldg(C.ux_n + c);
    S.pUy = __ldg(C.uy_n + c);
  }
}

// Prefetch ring: slot row & 7 of the four planes (T, rho, u_x, u_y).
#define PFW(plane, row, col) s_walk[EW_OFF_PF + ((plane) * EW_RPF + ((row) & (EW_RPF - 1))) * EW_W + (col)]

// Start the copies of row `row` (clamped to the lattice: the ghost rows above
// it repeat row ny - 1) into its prefetch slot; rows below the lattice are not
// read.  With 16-byte rows (nx a multiple of 4) the CTA's 64 threads copy the
// 4 planes x 64 frame columns as 64 pieces of 4 columns, one per thread (a
// piece starts on a multiple of 4 and never straddles the periodic edge);
// otherwise each thread copies its own column of the 4 planes.  Every call
// commits one group, empty or not, so that the groups of the rows in flight
// stay counted.
template <bool VEC>
__device__ __forceinline__ void walk_fetch(const StepArgs& A, const WalkCtx& C, int row) {
  if (row >= 0) {
    const int gr = row < A.ny ? row : A.ny - 1;
    if constexpr (VEC) {
      const int dst = (C.i >> 4) * EW_RPF * EW_W + 4 * (C.i & 15);  // plane i / 16, columns 4 (i % 16) ..
      cp_async16(&s_walk[EW_OFF_PF + dst + (row & (EW_RPF - 1)) * EW_W], C.vsrc + gr * A.nx);
    } else {
      const int c = gr * A.nx + C.gx;
      cp_async4(&PFW(0, row, C.i), C.T_in + c);
      cp_async4(&PFW(1, row, C.i), C.rho_n + c);
      cp_async4(&PFW(2, row, C.i), C.ux_n + c);
      cp_async4(&PFW(3, row, C.i), C.uy_n + c);
    }
  }
  cp_async_commit();
}

// Row `row` from its prefetch slot, with the substitutions of walk_load: zeros
// below the lattice, the wall temperature on Dirichlet rows, no rho or u on
// solid rows.  The slot's copies (made by other threads) completed before the
// last barrier of the previous walk step (walk_step waits for them there).
template <bool STEADY, int PF>
__device__ __forceinline__ void walk_take(const StepArgs& A, const WalkCtx& C, WalkState& S, int row) {
  const float T = PFW(0, row, C.i), R = PFW(1, row, C.i), U = PFW(2, row, C.i), V = PFW(3, row, C.i);
  if (STEADY) {
    S.pT = T;
    S.pR = R;
    S.pUx = U;
    S.pUy = V;
    return;
  }
  const Geo g = make_geo(A);
  const int gr = row < A.ny ? row : A.ny - 1;
  const bool below = row < 0, solid = !below && g.solid_row(gr);
  S.pT = below ? 0.f : (g.dirichlet_row(gr) ? (gr == 0 ? A.T_bottom : A.T_top) : T);
  S.pR = below || solid ? 0.f : R;
  S.pUx = below || solid ? 0.f : U;
  S.pUy = below || solid ? 0.f : V;
}

#define SW(off, slot, col) s_walk[(off) + (slot) * EW_W + (col)]

enum { WALK_GENERAL = 0, WALK_FILL = 1, WALK_STEADY = 2 };

// One walk step.  MODE WALK_STEADY: an interior segment past its first eight steps:
// every phase is active and no row of the step is solid, Dirichlet, a ghost,
// a wall-flux row or the top row, so all row tests compile away.  PF > 0: row r
// comes from the prefetch ring and row r + PF is fetched; PF = 0: row r was
// prefetched into S.p* and row r + 1 is loaded into them.
template <int P, int MODE, int PF, bool VEC>
__device__ __forceinline__ void walk_step(const StepArgs& A, const WalkCtx& C, WalkState& S, int t) {
  // RANGE: the segment's row-range tests; BND: the boundary rows' tests
  constexpr bool RANGE = MODE != WALK_STEADY, BND = MODE == WALK_GENERAL;
  constexpr int P0 = P & 3, P1 = (P + 3) & 3, P2 = (P + 2) & 3, P3 = (P + 1) & 3;  // rows r, r-1, r-2, r-3
  const Geo g = make_geo(A);
  const int ny = A.ny, W = A.W;
  const int i = C.i, ie = C.ie, iw = C.iw;
  const float dt = A.dt;
  const int r = t;
  auto wall_lam = [&](int row) -> float { return g.top_wall && row == ny - 1 ? A.lambda_top : A.lambda_w; };

  // ---- load phase: row r (prefetched) into the rings; prefetch row r + 1
  // (PF = 0: into registers) or start the copies of row r + PF (PF > 0)
  {
    if constexpr (PF > 0) {
      walk_take<!BND, PF>(A, C, S, r);
      walk_fetch<VEC>(A, C, r + PF);
    }
    float lam;
    if (!BND) {
      lam = S.pR * A.cvk;
    } else {
      const int gr = r < ny ? r : ny - 1;
      const bool solid = r >= 0 && g.solid_row(gr);
      lam = r < 0 ? A.lambda_w : (solid ? wall_lam(gr) : S.pR * A.cvk);
    }
    S.tn[P0] = S.pT;
    S.lam[P0] = lam;
    S.uy[P0] = S.pUy;
    SW(EW_OFF_TN, r & (EW_RTN - 1), i) = S.pT;
    SW(EW_OFF_UX, P0, i) = S.pUx;
    SW(EW_OFF_UY, P0, i) = S.pUy;
    SW(EW_OFF_LAM, P0, i) = lam;
    const float rho_r = S.pR;
    if constexpr (PF == 0) walk_load<!BND>(A, C, S, r + 1);
    __syncthreads();
    S.dx[P0] = SW(EW_OFF_UX, P0, ie) - SW(EW_OFF_UX, P0, iw);
    S.sy[P0] = SW(EW_OFF_UY, P0, ie) + SW(EW_OFF_UY, P0, iw);
    // ---- coefficients of row y = r - 1 (ring 3 of the segment)
    const int y = r - 1;
    if (!RANGE || (y >= C.ys - 3 && y < C.ye + 3 && y >= 0 && y < ny)) {
      float* cf = S.cf[P1];
#pragma unroll
      for (int q = 0; q < NCOEF; ++q) cf[q] = 0.f;
      const bool ysolid = BND && g.solid_row(y);
      S.rcv[P1] = ysolid ? A.rcv_w : S.rho1 * A.cv;
      const float l = S.lam[P1];
      const float lS = (!BND || y > 0) ? S.lam[P2] : l;
      if (BND) S.qf[P1] = y == ny - 2 ? harm(l, S.lam[P0]) : harm(l, lS);
      if (!BND || !g.dirichlet_row(y)) {
        // lambda_f / (rho cv) = 2 kd lambda_nb / (lambda + lambda_nb), kd = lambda / (rho cv) of the row
        const float kd = ysolid ? l * A.inv_rcv_w : A.kd;
        const float lE = SW(EW_OFF_LAM, P1, ie), lW = SW(EW_OFF_LAM, P1, iw);
        const float lN = (BND && g.top_open && y == ny - 1) ? l : S.lam[P0];
        const float cE = 2.f * kd * lE / (l + lE), cW = 2.f * kd * lW / (l + lW);
        const float cN = 2.f * kd * lN / (l + lN);
        // row 0 under an imposed flux: no conductive flux through its bottom face
        const float cS = (BND && y == 0) ? 0.f : 2.f * kd * lS / (l + lS);
        if (ysolid) {
          cf[C_AE] = cE;
          cf[C_AW] = cW;
          cf[C_AN] = cN;
          cf[C_AS] = cS;
        } else {
          const float ux = SW(EW_OFF_UX, P1, i), uy = S.uy[P1];
          const float divu = S.dx[P1] * (1.f / 3.f) + (S.dx[P0] + S.dx[P2]) * (1.f / 12.f) +
                             (S.uy[P0] - S.uy[P2]) * (1.f / 3.f) + (S.sy[P0] - S.sy[P2]) * (1.f / 12.f);
          const float br = A.b * S.rho1;
          cf[C_AE] = fmaf(ux, -1.f / 3.f, cE);
          cf[C_AW] = fmaf(ux, 1.f / 3.f, cW);
          cf[C_AN] = fmaf(uy, -1.f / 3.f, cN);
          cf[C_AS] = fmaf(uy, 1.f / 3.f, cS);
          cf[C_P] = (ux + uy) * (1.f / 12.f);
          cf[C_Q] = (ux - uy) * (1.f / 12.f);
          cf[C_AS_T] = divu * (A.R / A.cv) / (1.f - br);
          cf[C_BS] = divu * (A.a * A.kappa / A.cv) * S.rho1 / fmaf(br, 2.f - br, 1.f);
        }
      }
    }
    S.rho1 = rho_r;
  }

  // q_bottom (face 0|1), q_interface (face W-1|W) and q_top (face ny-2|ny-1 under
  // a top wall) accumulate the RK-weighted conductive flux of every stage
  auto wall_flux = [&](int y, float wk, float qf, float TS, float Tp, float TN) {
    if (!BND || !C.own_col) return;
    if (y == 1) ff_add(S.qbh, S.qbl, wk * qf * (TS - Tp));
    if (y == W) ff_add(S.qih, S.qil, wk * qf * (TS - Tp));
    if (g.top_wall && y == ny - 2) ff_add(S.qth, S.qtl, wk * qf * (Tp - TN));
  };
  auto special = [&](int y) -> bool {
    return BND && (y == 1 || y == W || (g.top_wall && y == ny - 2) || (y == 0 && g.bottom_flux));
  };
  const float qc = A.q_in * A.inv_rcv_w;

  // ---- stage 1 at y = r - 1: T^n at rows r - 2 .. r
  {
    const int y = r - 1;
    if (!RANGE || (y >= C.ys - 3 && y < C.ye + 3 && y >= 0)) {
      float v;
      if (!BND || y < ny) {
        const int lo = EW_OFF_TN + ((r - 2) & (EW_RTN - 1)) * EW_W, mid = EW_OFF_TN + ((r - 1) & (EW_RTN - 1)) * EW_W,
                  hi = EW_OFF_TN + (r & (EW_RTN - 1)) * EW_W;
        const float Tp = S.tn[P1];
        const float TS = (!BND || y > 0) ? S.tn[P2] : Tp;
        const float TN = S.tn[P0];
        float kk = walk_K(A, S.cf[P1], Tp, s_walk[mid + ie], s_walk[mid + iw], TN, TS, s_walk[hi + ie],
                          s_walk[hi + iw], s_walk[lo + ie], s_walk[lo + iw]);
        if (special(y)) {
          if (y == 0 && g.bottom_flux) kk += qc;
          wall_flux(y, dt * (1.f / 6.f), S.qf[P1], TS, Tp, TN);
        }
        S.acc[P1] = kk;
        v = fmaf(0.5f * dt, kk, Tp);
      } else {
        v = S.t1[P2];  // zero-gradient ghost above an open top: row ny - 1
      }
      S.t1[P1] = v;
      SW(EW_OFF_T1, P1, i) = v;
    }
  }
  __syncthreads();

  // ---- stage 2 at y = r - 2: T1 at rows r - 3 .. r - 1
  {
    const int y = r - 2;
    if (!RANGE || (y >= C.ys - 2 && y < C.ye + 2 && y >= 0)) {
      float v;
      if (!BND || y < ny) {
        const int lo = EW_OFF_T1 + P3 * EW_W, mid = EW_OFF_T1 + P2 * EW_W, hi = EW_OFF_T1 + P1 * EW_W;
        const float Tp = S.t1[P2];
        const float TS = (!BND || y > 0) ? S.t1[P3] : Tp;
        const float TN = S.t1[P1];
        float kk = walk_K(A, S.cf[P2], Tp, s_walk[mid + ie], s_walk[mid + iw], TN, TS, s_walk[hi + ie],
                          s_walk[hi + iw], s_walk[lo + ie], s_walk[lo + iw]);
        if (special(y)) {
          if (y == 0 && g.bottom_flux) kk += qc;
          wall_flux(y, dt * (2.f / 6.f), S.qf[P2], TS, Tp, TN);
        }
        S.acc[P2] = fmaf(2.f, kk, S.acc[P2]);
        v = fmaf(0.5f * dt, kk, S.tn[P2]);
      } else {
        v = S.t2[P3];
      }
      S.t2[P2] = v;
      SW(EW_OFF_T2, P2, i) = v;
    }
  }
  __syncthreads();

  // ---- stage 3 at y = r - 3: T2 at rows r - 4 .. r - 2
  {
    const int y = r - 3;
    if (!RANGE || (y >= C.ys - 1 && y < C.ye + 1 && y >= 0)) {
      float v;
      if (!BND || y < ny) {
        const int lo = EW_OFF_T2 + P0 * EW_W, mid = EW_OFF_T2 + P3 * EW_W, hi = EW_OFF_T2 + P2 * EW_W;
        const float Tp = S.t2[P3];
        const float TS = (!BND || y > 0) ? S.t2[P0] : Tp;
        const float TN = S.t2[P2];
        float kk = walk_K(A, S.cf[P3], Tp, s_walk[mid + ie], s_walk[mid + iw], TN, TS, s_walk[hi + ie],
                          s_walk[hi + iw], s_walk[lo + ie], s_walk[lo + iw]);
        if (special(y)) {
          if (y == 0 && g.bottom_flux) kk += qc;
          wall_flux(y, dt * (2.f / 6.f), S.qf[P3], TS, Tp, TN);
        }
        S.acc[P3] = fmaf(2.f, kk, S.acc[P3]);
        v = fmaf(dt, kk, S.tn[P3]);
      } else {
        v = S.t3[P0];
      }
      S.t3[P3] = v;
      SW(EW_OFF_T3, P3, i) = v;
    }
  }
  // row r + 1's copies (this thread's) complete; after the barrier every
  // thread's are, and the next walk step takes the row
  if constexpr (PF > 0) cp_async_wait<PF - 1>();
  __syncthreads();

  // ---- stage 4 at y = r - 4: T3 at rows r - 5 .. r - 3; the new temperature
  {
    const int y = r - 4;
    if (!RANGE || (y >= C.ys && y < C.ye)) {
      const int lo = EW_OFF_T3 + P1 * EW_W, mid = EW_OFF_T3 + P0 * EW_W, hi = EW_OFF_T3 + P3 * EW_W;
      const float Tp = S.t3[P0];
      const float TS = (!BND || y > 0) ? S.t3[P1] : Tp;
      const float TN = S.t3[P3];
      float kk = walk_K(A, S.cf[P0], Tp, s_walk[mid + ie], s_walk[mid + iw], TN, TS, s_walk[hi + ie],
                        s_walk[hi + iw], s_walk[lo + ie], s_walk[lo + iw]);
      if (special(y)) {
        if (y == 0 && g.bottom_flux) kk += qc;
        wall_flux(y, dt * (1.f / 6.f), S.qf[P0], TS, Tp, TN);
      }
      if (C.own_col) {
        const float T0 = SW(EW_OFF_TN, y & (EW_RTN - 1), i);
        const float Tnew = T0 + dt * (1.f / 6.f) * (S.acc[P0] + kk);
        if (nonfinite(Tnew)) S.err |= ERR_NONFINITE;
        C.T_out[y * A.nx + C.gx] = Tnew;
        if (C.last) ff_add(S.eh, S.el, Tnew * S.rcv[P0]);
      }
    }
  }
}
#undef SW

// Walk of strip sx, segment sg (rows [sg L, sg L + L)) of one domain.
template <int PF, bool VEC>
__device__ __forceinline__ void energy_walk(const StepArgs& A, int L, int sx, int sg, int part, int s, int nsub) {
  static_assert(PF >= 0 && PF < EW_RPF, "prefetch depth within the prefetch ring");
  __shared__ float s_red[EW_W / 32][NEPART][2];
  __shared__ int s_err;
  WalkCtx C;
  const int NC = A.nx * A.ny;
  C.T_in = s == 1 ? A.T_in : substep_buffer(A, s - 1, nsub);
  C.T_out = substep_buffer(A, s, nsub);
  C.rho_n = A.mom;
  C.ux_n = A.mom + NC;
  C.uy_n = A.mom + 2 * NC;
  C.i = threadIdx.x;
  C.ie = C.i + 1 < EW_W ? C.i + 1 : C.i;  // frame-edge columns read themselves
  C.iw = C.i > 0 ? C.i - 1 : C.i;
  const int gxu = sx * EW_OUT - EW_H + C.i;
  C.gx = wrapx(gxu, A.nx);
  C.own_col = C.i >= EW_H && C.i < EW_H + EW_OUT && gxu < A.nx;
  C.ys = sg * L;
  C.ye = C.ys + L < A.ny ? C.ys + L : A.ny;
  C.last = s == nsub;
  if constexpr (VEC) {
    // thread i copies plane i / 16, frame columns 4 (i % 16) .. + 3: a piece
    // starts on a multiple of 4 columns and, nx being one too, never
    // straddles the periodic edge
    static_assert(EW_W == 4 * 16, "16-byte prefetch: four planes of sixteen 4-column pieces");
    const int plane = C.i >> 4, col = 4 * (C.i & 15);
    const float* base = plane == 0 ? C.T_in : (plane == 1 ? C.rho_n : (plane == 2 ? C.ux_n : C.uy_n));
    C.vsrc = base + wrapx(sx * EW_OUT - EW_H + col, A.nx);
  } else {
    C.vsrc = nullptr;
  }
  if (threadIdx.x == 0) s_err = 0;

  WalkState S;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    S.tn[q] = S.t1[q] = S.t2[q] = S.t3[q] = S.acc[q] = S.rcv[q] = S.qf[q] = 0.f;
    S.dx[q] = S.sy[q] = S.uy[q] = S.lam[q] = 0.f;
#pragma unroll
    for (int c = 0; c < NCOEF; ++c) S.cf[q][c] = 0.f;
  }
  S.rho1 = 0.f;
  S.eh = S.el = S.qbh = S.qbl = S.qih = S.qil = S.qth = S.qtl = 0.f;
  S.err = 0;
  // The stage rings of row -1 are read (times a zero coefficient) by row 0 of
  // the first segment but never written: start them at zero, not at whatever an
  // earlier kernel left in shared memory (a NaN there would survive 0 * NaN).
  // Each thread clears its own column; the first step's barrier orders these
  // stores before any read.
#pragma unroll
  for (int q = 0; q < 3 * EW_R; ++q) s_walk[EW_OFF_T1 + q * EW_W + C.i] = 0.f;
  const int t0 = C.ys - 4;  // a multiple of four: t & 3 is the unrolled phase
  if constexpr (PF == 0) {
    walk_load<false>(A, C, S, t0);
  } else {
#pragma unroll
    for (int k = 0; k < PF; ++k) walk_fetch<VEC>(A, C, t0 + k);
    cp_async_wait<PF - 1>();  // row t0, for the first walk step
    __syncthreads();
  }
  // Steps t .. t+3 touch rows t - 5 .. t + 4.  They run in the steady form when
  // every phase of each is active (t >= ys + 4, t + 3 < ye + 4) and those rows
  // are fluid rows at least two rows from the wall rows and three from the top
  // (no solid, Dirichlet, ghost, top or wall-flux row).
  // Groups whose rows are all such rows but not every phase is active (the
  // pipeline's fill at the segment's start) run WALK_FILL: the row-range tests
  // of the general form without its boundary-row tests.
  const int r_lo = A.W + 7, r_hi = A.ny - 7;
  const int t_lo = max(C.ys + 4, r_lo), t_hi = min(C.ye, r_hi);  // steady groups: t_lo <= t <= t_hi
  for (int t = t0; t < C.ye + 4; t += 4) {
    if (t >= t_lo && t <= t_hi) {
      walk_step<0, WALK_STEADY, PF, VEC>(A, C, S, t);
      walk_step<1, WALK_STEADY, PF, VEC>(A, C, S, t + 1);
      walk_step<2, WALK_STEADY, PF, VEC>(A, C, S, t + 2);
      walk_step<3, WALK_STEADY, PF, VEC>(A, C, S, t + 3);
    } else if (t >= r_lo && t <= r_hi) {
      walk_step<0, WALK_FILL, PF, VEC>(A, C, S, t);
      walk_step<1, WALK_FILL, PF, VEC>(A, C, S, t + 1);
      walk_step<2, WALK_FILL, PF, VEC>(A, C, S, t + 2);
      walk_step<3, WALK_FILL, PF, VEC>(A, C, S, t + 3);
    } else {
      walk_step<0, WALK_GENERAL, PF, VEC>(A, C, S, t);
      walk_step<1, WALK_GENERAL, PF, VEC>(A, C, S, t + 1);
      walk_step<2, WALK_GENERAL, PF, VEC>(A, C, S, t + 2);
      walk_step<3, WALK_GENERAL, PF, VEC>(A, C, S, t + 3);
    }
  }
  if constexpr (PF > 0) cp_async_wait<0>();  // copies of the rows past the walk: none left in flight at exit
  float ah[NEPART] = {S.qbh, S.qth, S.qih, S.eh}, al[NEPART] = {S.qbl, S.qtl, S.qil, S.el};
  if (S.err) atomicOr(&s_err, S.err);
  block_partials<EW_W, NEPART>(ah, al, s_red, A.epart + (long long)part * NEPART, s > 1);
  if (threadIdx.x == 0 && s_err) atomicOr(&A.state->error_flags, s_err);
}

template <int L, int MINB, int PF>
__global__ void __launch_bounds__(EW_W, MINB) k_energy_walk(const StepArgs A, int s, int nsub) {
  static_assert(L % 4 == 0, "segments start on a multiple of four rows");
  // 16-byte prefetch pieces where the rows allow them (nx a multiple of 4)
  if (PF > 0 && (A.nx & 3) == 0)
    energy_walk<PF, true>(A, L, blockIdx.x, blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x, s, nsub);
  else
    energy_walk<PF, false>(A, L, blockIdx.x, blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x, s, nsub);
}

template <int L, int MINB, int PF>
__global__ void __launch_bounds__(EW_W, MINB) k_energy_walk_batch(const StepArgs P, const DomArgs* __restrict__ desc,
                                                               const int2* __restrict__ blk,
                                                               const int* __restrict__ active, int s, int nsub) {
  static_assert(L % 4 == 0, "segments start on a multiple of four rows");
  __shared__ DomArgs sD;
  __shared__ int s_act;
  __shared__ int2 s_bl;
  __shared__ float2 s_lg;
  if (!batch_prologue<EW_W>(desc, blk, active, nullptr, sD, s_bl, s_lg, s_act)) return;
  StepArgs A = P;
  apply_dom(A, sD);
  const int local = s_bl.y;
  const int strips = (A.nx + EW_OUT - 1) / EW_OUT;
  if (PF > 0 && (A.nx & 3) == 0)
    energy_walk<PF, true>(A, L, local % strips, local / strips, local, s, nsub);
  else
    energy_walk<PF, false>(A, L, local % strips, local / strips, local, s, nsub);
}

}  // namespace hlb
