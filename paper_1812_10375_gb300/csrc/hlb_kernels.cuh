// Device code of the hybrid thermal LB phase-change step (Hu & Liu, arXiv 1812.10375).
//
// One launch of k_step advances one domain by one coupled step:
//   pull-streaming with halfway bounce-back and open-top rules (Eqs. 1-2,
//   Sections 3.3, 4.2) -> rho (Eq. 5) -> psi from the Peng-Robinson EOS
//   (Eqs. 7, 28) -> F = F_m + F_ads + F_b (Eqs. 6, 9, 10) -> u (Eq. 5) ->
//   MRT collision with Li's forcing (Eqs. 2-4, 8) and the RK4 update of the
//   energy equation (Eqs. 17-19) with finite-volume harmonic face
//   conductivities (Eqs. 22-26).
// The energy update of an output cell depends on u at distance 4 and hence on
// psi at distance 5 and the populations at distance 6, so each CTA recomputes
// a ring-6 halo of its tile in shared memory (reads of neighbouring tiles hit
// L2) and writes only its own tile: 36 B + 36 B of populations and 4 B + 4 B
// of temperature per cell from HBM.
#pragma once
#include "hlb_internal.cuh"

namespace hlb {

enum { TOP_WALL = 0, TOP_CONST_RHO = 1, TOP_CONVECTIVE = 2 };

constexpr int HALO = 6;       // frame halo of the fused kernel
// Compiled tile variants of the fused kernel (tile height TY, threads per CTA,
// CTAs per SM the register budget is sized for); the host autotuner picks one.
#define HLB_STEP_VARIANTS(X) X(28, 512, 2) X(16, 256, 3) X(20, 512, 2)

// x is at most a frame halo (plus a tile) outside [0, nx): fold it back
// with additions instead of an integer division.
__device__ __forceinline__ int wrapx(int x, int nx) {
  while (x < 0) x += nx;
  while (x >= nx) x -= nx;
  return x;
}

__device__ __forceinline__ bool nonfinite(float v) {
  return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u;
}

struct Geo {
  int nx, ny, W;
  bool top_wall, top_open, bottom_flux;
  __device__ __forceinline__ bool solid_row(int y) const { return y < W || (top_wall && y == ny - 1); }
  __device__ __forceinline__ bool dirichlet_row(int y) const {
    return (y == 0 && !bottom_flux) || (top_wall && y == ny - 1);
  }
};

__device__ __forceinline__ Geo make_geo(const StepArgs& A) {
  Geo g;
  g.nx = A.nx;
  g.ny = A.ny;
  g.W = A.W;
  g.top_wall = A.top_bc == TOP_WALL;
  g.top_open = A.top_bc != TOP_WALL;
  g.bottom_flux = A.bottom_flux != 0;
  return g;
}

// psi^2 = 2 (rho/3 - p_EOS) with p_EOS of Eq. (28); Eq. (7) with c = 1, G = -1.
__device__ __forceinline__ float pr_psi2(const StepArgs& A, float rho, float T) {
  const float sTr = sqrtf(fmaxf(T, 0.f) * A.invTc);
  const float al = 1.f + A.kappa * (1.f - sTr);
  const float br = A.b * rho;
  const float p = rho * A.R * T / (1.f - br) - A.a * al * al * rho * rho / (1.f + 2.f * br - br * br);
  return 2.f * (rho * (1.f / 3.f) - p);
}

// Post-streaming populations (deviation form) of fluid node (x, y): pull from
// x - e_i; halfway bounce-back where x - e_i is solid; populations entering an
// open top row from above are the rest equilibrium at rho_v (constant density)
// or the convective-outlet update with the lagged velocity U (Uc = U / (1 + U)).
// D2Q9 order: 0 rest, 1 (+x), 2 (+y), 3 (-x), 4 (-y), 5 (+x+y), 6 (-x+y), 7 (-x-y), 8 (+x-y).
// bb_s / sol_n: the rows below / above y are solid.
__device__ __forceinline__ void pull(const StepArgs& A, const Geo& g, int x, int xm, int xp, int y, bool bb_s,
                                     bool sol_n, float Uc, float f[9]) {
  const int nx = g.nx;
  const int P = (int)A.plane;  // 9 planes < 2^31 floats (checked at init)
  const float* __restrict__ F = A.f_in;
  const int r0 = y * nx;
  const int rs = r0 - nx;
  const int rn = r0 + nx;
  const bool open_n = g.top_open && y == g.ny - 1;
  const bool bb_n = !open_n && sol_n;
  f[0] = __ldg(F + r0 + x);
  f[1] = __ldg(F + 1 * P + r0 + xm);
  f[3] = __ldg(F + 3 * P + r0 + xp);
  if (bb_s) {
    f[2] = __ldg(F + 4 * P + r0 + x);
    f[5] = __ldg(F + 7 * P + r0 + x);
    f[6] = __ldg(F + 8 * P + r0 + x);
  } else {
    f[2] = __ldg(F + 2 * P + rs + x);
    f[5] = __ldg(F + 5 * P + rs + xm);
    f[6] = __ldg(F + 6 * P + rs + xp);
  }
  if (open_n) {
    if (A.top_bc == TOP_CONST_RHO) {
      const float d = A.rho_v - A.rho_ref;
      f[4] = d * (1.f / 9.f);
      f[7] = d * (1.f / 36.f);
      f[8] = d * (1.f / 36.f);
    } else {
      // f_i(top) = [f_i^{n-1}(top) + U f_i^n(top-1)] / (1 + U), evaluated as
      // prev + Uc (below - prev) with Uc = U / (1 + U) from FP64: in FP32, 1 + U
      // would keep only a few digits of U ~ 1e-5.  f_i^n(top-1) is pulled from this row.
      const float p4 = A.ftop_in[x], p7 = A.ftop_in[nx + x], p8 = A.ftop_in[2 * nx + x];
      f[4] = p4 + Uc * (__ldg(F + 4 * P + r0 + x) - p4);
      f[7] = p7 + Uc * (__ldg(F + 7 * P + r0 + xp) - p7);
      f[8] = p8 + Uc * (__ldg(F + 8 * P + r0 + xm) - p8);
    }
  } else if (bb_n) {
    f[4] = __ldg(F + 2 * P + r0 + x);
    f[7] = __ldg(F + 5 * P + r0 + x);
    f[8] = __ldg(F + 6 * P + r0 + x);
  } else {
    f[4] = __ldg(F + 4 * P + rn + x);
    f[7] = __ldg(F + 7 * P + rn + xp);
    f[8] = __ldg(F + 8 * P + rn + xm);
  }
}

__device__ __forceinline__ float sum9(const float f[9]) {
  return ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
}

// MRT collision with Li's forcing, Eqs. (2)-(4), (8), on deviation populations
// f~ = f - w rho_ref; moments m~ = M f~ differ from m = M f by rho_ref (1, -2, 1, 0, ...).
// Applied as an increment f* = f + M^-1 dm with dm = -Lambda (m - m_eq) + (I - Lambda/2) S:
// the density row of dm is 0 and the momentum rows are exactly F (because
// j - rho u = -F/2 by Eq. 5), so no rounded 1/9 or 1/6 multiplies rho or j and
// FP32 rounding cannot bias mass or momentum from step to step.
// Fm2_psi2 = |F_m|^2 / psi^2.  Writes the nine post-collision values and returns
// a sum of the density moment and the moment increments, non-finite whenever
// an input population or an increment is.
__device__ __forceinline__ float collide_store(const StepArgs& A, const float f[9], float rho, float ux, float uy,
                                               float Fx, float Fy, float Fm2_psi2, int off) {
  // the moments share their partial sums: axis pairs (1,3), (2,4) and
  // diagonal pairs (5,7), (6,8)
  const float s13 = f[1] + f[3], s24 = f[2] + f[4], s57 = f[5] + f[7], s68 = f[6] + f[8];
  const float d57 = f[5] - f[7], d68 = f[6] - f[8];
  const float sa = s13 + s24;
  const float sd = s57 + s68;
  const float m0 = f[0] + sa + sd;  // rho - rho_ref
  const float me = -4.f * f[0] - sa + 2.f * sd;
  const float mz = 4.f * f[0] - 2.f * sa + sd;
  const float ax = f[1] - f[3], ay = f[2] - f[4];
  const float cx = d57 - d68;
  const float cy = d57 + d68;
  const float qx = -2.f * ax + cx;
  const float qy = -2.f * ay + cy;
  const float pxx = s13 - s24;
  const float pxy = s57 - s68;

  const float u2 = ux * ux + uy * uy;
  const float uF = ux * Fx + uy * Fy;
  float tau = A.tau_v + (rho - A.rho_v) * A.dtau_drho;
  tau = fminf(fmaxf(tau, fminf(A.tau_l, A.tau_v)), fmaxf(A.tau_l, A.tau_v));
  const float snu = 1.f / tau;

  const float de = -A.s_e * (me + 2.f * m0 - 3.f * rho * u2) + (1.f - 0.5f * A.s_e) * (6.f * uF) + A.sig_e * Fm2_psi2;
  const float dz = -A.s_z * (mz - m0 + 3.f * rho * u2) - (1.f - 0.5f * A.s_z) * (6.f * uF) - A.sig_z * Fm2_psi2;
  const float dqx = -A.s_q * (qx + rho * ux) - (1.f - 0.5f * A.s_q) * Fx;
  const float dqy = -A.s_q * (qy + rho * uy) - (1.f - 0.5f * A.s_q) * Fy;
  const float dpxx = -snu * (pxx - rho * (ux * ux - uy * uy)) + (1.f - 0.5f * snu) * 2.f * (ux * Fx - uy * Fy);
  const float dpxy = -snu * (pxy - rho * ux * uy) + (1.f - 0.5f * snu) * (ux * Fy + uy * Fx);

  // M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4); the density component is 0
  const float r1 = de * (1.f / 36.f), r2 = dz * (1.f / 36.f);
  const float r3 = Fx * (1.f / 6.f), r4 = dqx * (1.f / 12.f);
  const float r5 = Fy * (1.f / 6.f), r6 = dqy * (1.f / 12.f);
  const float r7 = dpxx * 0.25f, r8 = dpxy * 0.25f;
  const float ba = -r1 - 2.f * r2;
  const float bd = 2.f * r1 + r2;
  // increments of opposite directions share their even and odd parts
  const float ex = ba + r7, ox = r3 - 2.f * r4;  // directions 1 and 3
  const float ey = ba - r7, oy = r5 - 2.f * r6;  // directions 2 and 4
  const float cxq = r3 + r4, cyq = r5 + r6;
  const float ep = bd + r8, em = bd - r8;
  const float op = cxq + cyq, om = cyq - cxq;  // directions 5/7 and 6/8
  const float o0 = f[0] + (4.f * (r2 - r1));
  const float o1 = f[1] + (ex + ox);
  const float o2 = f[2] + (ey + oy);
  const float o3 = f[3] + (ex - ox);
  const float o4 = f[4] + (ey - oy);
  const float o5 = f[5] + (ep + op);
  const float o6 = f[6] + (em + om);
  const float o7 = f[7] + (ep - op);
  const float o8 = f[8] + (em - om);
  const int P = (int)A.plane;
  float* __restrict__ out = A.f_out + off;
  out[0] = o0;
  out[P] = o1;
  out[2 * P] = o2;
  out[3 * P] = o3;
  out[4 * P] = o4;
  out[5 * P] = o5;
  out[6 * P] = o6;
  out[7 * P] = o7;
  out[8 * P] = o8;
  // non-finite check: every output is f_i plus a combination of these
  return (m0 + de) + (dz + dqx) + (dqy + dpxx) + dpxy;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Compensated (float-float) summation: hi + lo carries about twice the
// precision of FP32, so the per-block partial sums stay accurate to ~1e-14
// relative while all arithmetic runs in the FP32 pipes (GB300's FP64 pipe
// runs at 1/64 of the FP32 rate).  TwoSum is exact in round-to-nearest.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}

__device__ __forceinline__ void ff_merge(float& hi, float& lo, float h2, float l2) {
  ff_add(hi, lo, h2);
  lo += l2;
  const float s = hi + lo;  // renormalise (|hi| >= |lo|)
  lo = lo - (s - hi);
  hi = s;
}

__device__ __forceinline__ void ff_warp_sum(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
    ff_merge(hi, lo, h2, l2);
  }
}

// Geometry of the fused kernel's tile: a frame of FRAME_W = 64 columns (the
// TILE_W = 52 output columns plus a 6-cell halo on either side) by TY + 12 rows.
// Each thread owns one frame column (tid & 63) for the whole step and visits
// every NPH-th frame row (NPH = threads / 64, starting at tid >> 6), so a warp
// always works on 32 consecutive cells of one row: x-wrapping and the wetting
// table are resolved once per thread and row properties are uniform across a
// warp.
constexpr int FRAME_W = 64;
constexpr int TILE_W = FRAME_W - 2 * HALO;

// Ten frame arrays; during passes A and B the last five of them (and a tail
// beyond them where needed) hold the tile's post-streaming populations.
template <int TY>
constexpr int step_smem_floats() {
  constexpr int fn = FRAME_W * (TY + 2 * HALO);
  constexpr int frames = 10 * fn, stash = 5 * fn + 9 * TY * TILE_W;
  return frames > stash ? frames : stash;
}

// Bit m of byte k of a row-flag word describes the thread's m-th frame row.
__device__ __forceinline__ bool rowbit(unsigned w, int k, int m) { return (w >> (8 * k + m)) & 1u; }

// Fused coupled step on tile (bx, by).  Ring r of the tile = frame cells within
// distance r of the tile.  `part` is the tile's slot in the partial-sum array.
// Uc, rho_ave: the lagged outlet factor U/(1+U) and mean density of the domain.
// INT: the tile is interior (tile_interior below): every frame row is a fluid
// row at least one row away from a solid row and from the top two rows, so the
// row-class tests (solid, Dirichlet, bounce-back, open top, wall-flux and
// diagnostic rows, ghost rows) are known to be false and compile away.
// ISO: the energy equation's diffusion term in the isotropic central form of
// Eq. (21), lambda lap(T) + grad(lambda) . grad(T) with the Laplacian of
// Eq. (20) and the gradients of Eq. (19), instead of the finite-volume faces.
template <int TY, int NTHREADS, bool INT, bool ISO = false>
__device__ __forceinline__ void step_tile(const StepArgs& A, int bx, int by, int part, float* sm, float Uc,
                                          float rho_ave) {
  constexpr int H = HALO, TX = TILE_W, FW = FRAME_W, FH = TY + 2 * H, FN = FW * FH;
  constexpr int NPH = NTHREADS / FW;  // row phases
  constexpr int NJ = FH / NPH;
  constexpr int TSZ = TY * TX;
  static_assert(NTHREADS % FW == 0, "one thread per frame column and row phase");
  static_assert(FH % NPH == 0, "frame height must be a multiple of the row phases");
  static_assert(NJ <= 8, "row flags hold eight rows per byte");
  float* const sT0 = sm;            // T^n, ring 5
  float* const sRho = sm + FN;      // rho, ring 5      -> stage buffer Ta
  float* const sPsi = sm + 2 * FN;  // psi, ring 5      -> east-face conductivity
  float* const sUx = sm + 3 * FN;   // u, ring 4
  float* const sUy = sm + 4 * FN;
  float* const sTb = sm + 5 * FN;   // stage buffer Tb
  float* const sLan = sm + 6 * FN;  // north-face conductivity
  float* const sIrcv = sm + 7 * FN; // 1/(rho cv), ring 3
  float* const sAs = sm + 8 * FN;   // latent-heat source coefficients, ring 3
  float* const sBs = sm + 9 * FN;
  float* const sF = sm + 5 * FN;    // passes A-B: populations of the tile, 9 planes of TSZ
  float* const sLae = sPsi;
  float* const sTa = sRho;
  __shared__ int s_err;
  __shared__ float s_red[NTHREADS / 32][NPART][2];
  // Wall-flux partials (q_bottom, q_top, q_interface) per frame column as
  // compensated (hi, lo): each lies on one lattice row, so one thread owns each
  // entry and no register carries it through the stages.
  __shared__ float s_q[3][2][FW];

  const Geo g = make_geo(A);
  const int nx = A.nx, ny = A.ny;
  const int x0 = bx * TX, y0 = by * TY;
  const int tid = threadIdx.x;
  const int i = tid & (FW - 1), jp = tid >> 6;
  // Frame rows above the lattice's top row (gy >= ny) hold copies of that row
  // (the zero-gradient ghost of an open top; unused above a top wall), so
  // every stencil reads its north and south neighbours at fixed offsets.
  const int jtop = ny - 1 - y0 + H;  // frame row of gy = ny - 1
  const bool has_ghost = !INT && jtop < FH - 1;
  auto fill_ghost = [&](float* a) {
    for (int j = jtop + 1 + jp; j < FH; j += NPH) a[j * FW + i] = a[jtop * FW + i];
  };
  const int gxu = x0 - H + i;
  const int gx = wrapx(gxu, nx);
  const int xm = gx == 0 ? nx - 1 : gx - 1;
  const int xp = gx == nx - 1 ? 0 : gx + 1;
  const float gw = __ldg(A.Gw + gx);
  const bool own_col = i >= H && i < H + TX && gxu < nx;
  // Row flags of the thread's frame rows j = jp + NPH m for passes A and B,
  // built once from prefix masks.  rf byte 0: a lattice row within distance 4
  // of the tile; byte 1: within distance 5 (passes A and B evaluate every
  // column of such rows, so their loops stay warp-uniform; columns outside the
  // ring are never read later); byte 2: an output cell of this tile; byte 3: a
  // row that carries a diagnostic (gy = 1, W, ny - 2, ny - 1).  fl byte 0:
  // solid row; 1: Dirichlet row; 2: row below solid; 3: row above solid (the
  // row index clamped to the lattice, as the ghost rows are).
  static_assert(NPH == 4 || NPH == 8 || NPH == 16, "row phases must be a power of two");
  constexpr int SH = NPH == 4 ? 2 : (NPH == 8 ? 3 : 4);
  constexpr unsigned ALL = (1u << NJ) - 1u;
  const int g0 = y0 - H + jp;  // lattice row of the thread's first frame row
  // masks of the thread's rows with gy < v and with frame row j < v
  auto lt = [&](int v) -> unsigned { return (1u << min(max((v - g0 + NPH - 1) >> SH, 0), NJ)) - 1u; };
  auto ltj = [&](int v) -> unsigned { return (1u << min(max((v - jp + NPH - 1) >> SH, 0), NJ)) - 1u; };
  auto eq = [&](int v) -> unsigned { return lt(v + 1) & ~lt(v); };
  const unsigned lat = INT ? ALL : lt(ny) & ~lt(0);
  const unsigned ring4 = ltj(H + TY + 4) & ~ltj(H - 4) & lat;
  const unsigned ring5 = ltj(H + TY + 5) & ~ltj(H - 5) & lat;
  const unsigned ownr = own_col ? ltj(H + TY) & ~ltj(H) & lat : 0u;
  const unsigned diag = INT ? 0u : eq(1) | eq(A.W) | eq(ny - 2) | eq(ny - 1);
  const bool tw = g.top_wall;
  const unsigned solid = lt(A.W) | (tw ? ALL & ~lt(ny - 1) : 0u);      // solid_row(min(gy, ny - 1))
  const unsigned dirich = (g.bottom_flux ? 0u : eq(0)) | (tw ? eq(ny - 1) : 0u);  // dirichlet_row(gy)
  const unsigned sol_below = lt(A.W + 1) | (tw ? eq(ny) : 0u);          // solid_row(gy - 1)
  const unsigned sol_above = lt(A.W - 1) | (tw ? ALL & ~lt(ny - 2) : 0u);  // solid_row(min(gy + 1, ny - 1))
  const unsigned rf = ring4 | ring5 << 8 | ownr << 16 | diag << 24;
  const unsigned fl = INT ? 0u : solid | dirich << 8 | sol_below << 16 | sol_above << 24;
  if (tid == 0) s_err = 0;  // read after the barriers below
  for (int t = tid; t < 3 * 2 * FW; t += NTHREADS) (&s_q[0][0][0])[t] = 0.f;
  int err = 0;
  // Diagnostics partial sums in compensated FP32 (hi, lo); one thread converts
  // the block's six totals to FP64.
  float ah[NPART], al[NPART];
#pragma unroll
  for (int q = 0; q < NPART; ++q) ah[q] = al[q] = 0.f;

  // ---- pass A (ring 5): T^n, rho and psi; the tile's own populations are stashed.
  // This pass waits on L2 and HBM: rows go in pairs whose loads are all issued
  // before either row is used, which doubles the loads in flight per thread.
  // interior rows (no solid row next to them, not the open top row) pull at
  // fixed offsets from one row pointer
  const int P = (int)A.plane;
  const int o1 = P + xm - gx, o3 = 3 * P + xp - gx;
  const int o2 = 2 * P - nx, o5 = 5 * P - nx + xm - gx, o6 = 6 * P - nx + xp - gx;
  const int o4 = 4 * P + nx, o7 = 7 * P + nx + xp - gx, o8 = 8 * P + nx + xm - gx;
  auto fetch = [&](int m, float f[9]) -> float {
    const int gy = y0 - H + jp + NPH * m;
    const int c = gy * nx + gx;
    const float T = rowbit(fl, 1, m) ? (gy == 0 ? A.T_bottom : A.T_top) : __ldg(A.T_in + c);
    if (!rowbit(fl, 0, m)) {
      const bool sol_s = rowbit(fl, 2, m), sol_n = rowbit(fl, 3, m);
      if (INT || (!sol_s && !sol_n && !(g.top_open && gy == ny - 1))) {
        const float* __restrict__ F = A.f_in + c;
        f[0] = __ldg(F);
        f[1] = __ldg(F + o1);
        f[3] = __ldg(F + o3);
        f[2] = __ldg(F + o2);
        f[5] = __ldg(F + o5);
        f[6] = __ldg(F + o6);
        f[4] = __ldg(F + o4);
        f[7] = __ldg(F + o7);
        f[8] = __ldg(F + o8);
      } else {
        pull(A, g, gx, xm, xp, gy, sol_s, sol_n, Uc, f);
      }
    }
    return T;
  };
  auto settle = [&](int m, const float f[9], float T) {
    const int j = jp + NPH * m;
    const int idx = j * FW + i;
    sT0[idx] = T;
    if (rowbit(fl, 0, m)) {  // solid row: no populations
      sRho[idx] = 0.f;
      sPsi[idx] = 0.f;
      return;
    }
    const float rho = A.rho_ref + sum9(f);
    float p2 = pr_psi2(A, rho, A.eos_T_fixed ? A.Ts : T);
    if (!(p2 >= 0.f)) {
      err |= ERR_PSI_NEG;
      p2 = 0.f;
    }
    sRho[idx] = rho;
    sPsi[idx] = sqrtf(p2);
    // momentum sum e_i f_i of ring-4 cells, parked in the velocity arrays
    // (pass B replaces it in place by u, so halo cells need no second pull)
    if (rowbit(rf, 0, m)) {
      sUx[idx] = (f[1] - f[3]) + ((f[5] - f[6]) - (f[7] - f[8]));
      sUy[idx] = (f[2] - f[4]) + ((f[5] + f[6]) - (f[7] + f[8]));
    }
    if (rowbit(rf, 2, m)) {
      const int c = (j - H) * TX + (i - H);
#pragma unroll
      for (int q = 0; q < 9; ++q) sF[q * TSZ + c] = f[q];
    }
  };
#pragma unroll 1
  for (unsigned mm = (rf >> 8) & 0xffu; mm;) {
    const int m1 = __ffs(mm) - 1;
    mm &= mm - 1;
    float f1[9], f2[9];
    const float T1 = fetch(m1, f1);
    if (mm) {
      const int m2 = __ffs(mm) - 1;
      mm &= mm - 1;
      const float T2 = fetch(m2, f2);
      settle(m1, f1, T1);
      settle(m2, f2, T2);
    } else {
      settle(m1, f1, T1);
    }
  }
  __syncthreads();
  if (has_ghost) {
    fill_ghost(sT0);
    fill_ghost(sRho);
    fill_ghost(sPsi);
    __syncthreads();
  }

  // ---- pass B (ring 4): forces and velocity; collide the tile
#pragma unroll 1
  for (unsigned mm = rf & 0xffu; mm; mm &= mm - 1) {
    const int m = __ffs(mm) - 1;
    const int j = jp + NPH * m;
    const int idx = j * FW + i;
    if (rowbit(fl, 0, m)) {
      sUx[idx] = 0.f;
      sUy[idx] = 0.f;
      continue;
    }
    const float psi = sPsi[idx], rho = sRho[idx];
    const int js = j - 1, jn = j + 1;
    const bool sol_s = rowbit(fl, 2, m);
    const bool sol_n = rowbit(fl, 3, m);
    // Eq. (6); a solid neighbour carries psi(x)
    const float pE = sPsi[idx + 1], pW = sPsi[idx - 1];
    const float pN = sol_n ? psi : sPsi[jn * FW + i];
    const float pS = sol_s ? psi : sPsi[js * FW + i];
    const float pNE = sol_n ? psi : sPsi[jn * FW + i + 1];
    const float pNW = sol_n ? psi : sPsi[jn * FW + i - 1];
    const float pSE = sol_s ? psi : sPsi[js * FW + i + 1];
    const float pSW = sol_s ? psi : sPsi[js * FW + i - 1];
    const float sx = (pE - pW) * (1.f / 3.f) + ((pNE - pNW) + (pSE - pSW)) * (1.f / 12.f);
    const float sy = (pN - pS) * (1.f / 3.f) + ((pNE + pNW) - (pSE + pSW)) * (1.f / 12.f);
    const float Fmx = -A.G * psi * sx;
    const float Fmy = -A.G * psi * sy;
    // Eq. (10) with weights omega/3: solid rows are whole rows, so only a
    // normal component (1/9 + 2/36) (s_N - s_S) remains
    const float Fay = gw * psi * psi * ((float)sol_n - (float)sol_s) * (1.f / 6.f);
    const float Fx = Fmx;
    const float Fy = Fmy + Fay + (rho - rho_ave) * A.g_y;  // Eq. (9)
    const float irho = 1.f / rho;
    const float ux = (sUx[idx] + 0.5f * Fx) * irho;
    const float uy = (sUy[idx] + 0.5f * Fy) * irho;
    sUx[idx] = ux;
    sUy[idx] = uy;
    if (rowbit(rf, 2, m)) {
      const int gy = y0 - H + j;
      const int c = (j - H) * TX + (i - H);
      float f[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) f[q] = sF[q * TSZ + c];
      const float fsum = collide_store(A, f, rho, ux, uy, Fx, Fy, A.G * A.G * (sx * sx + sy * sy), gy * nx + gx);
      if (nonfinite(fsum)) err |= ERR_NONFINITE;
      ff_add(ah[P_MASS], al[P_MASS], rho);
      if (rowbit(rf, 3, m)) {
        if (gy == A.W && rho < A.rho_mid) ff_add(ah[P_VCOV], al[P_VCOV], 1.f);
        if (gy == ny - 2) ff_add(ah[P_UTOP], al[P_UTOP], uy);
        if (A.top_bc == TOP_CONVECTIVE && gy == ny - 1) {
          A.ftop_out[gx] = f[4];
          A.ftop_out[nx + gx] = f[7];
          A.ftop_out[2 * nx + gx] = f[8];
        }
      }
    }
  }
  // the pass-B partial sums are complete: reduce them over the warp now so that
  // their registers are free during the energy stages
  const int lane = tid & 31, warp = tid >> 5;
  auto warp_flush = [&](int q) {
    // wall- and top-row quantities are zero in most warps: skip their reduction there
    if (__any_sync(0xffffffffu, ah[q] != 0.f || al[q] != 0.f)) ff_warp_sum(ah[q], al[q]);
    if (lane == 0) {
      s_red[warp][q][0] = ah[q];
      s_red[warp][q][1] = al[q];
    }
  };
  warp_flush(P_MASS);
  warp_flush(P_VCOV);
  warp_flush(P_UTOP);
  __syncthreads();
  if (has_ghost) {
    fill_ghost(sUx);
    fill_ghost(sUy);
    __syncthreads();
  }

  // ---- pass C: face conductivities (Eq. 25) on the rows of ring 4, coefficients
  // on the rows of ring 3 (every column, as in the stages); lambda = rho cv k in
  // the fluid (Section 2.2), lambda_w in solid rows
  const float lam_w = A.lambda_w, cvk = A.cvk;
  // conductivity of a solid row: the heater's, or the top wall's (Section 3.2)
  auto wall_lam = [&](int row) -> float { return g.top_wall && row == ny - 1 ? A.lambda_top : lam_w; };
#pragma unroll
  for (int m = 0; m < NJ; ++m) {
    const int j = jp + NPH * m;
    const int gy = y0 - H + j;
    if (j < H - 4 || j >= H + TY + 4 || (!INT && (gy < 0 || gy >= ny))) continue;
    const int idx = j * FW + i;
    const bool solid = !INT && g.solid_row(gy);
    const float lam = solid ? wall_lam(gy) : sRho[idx] * cvk;
    {
      const float le = solid ? wall_lam(gy) : sRho[idx + 1] * cvk;
      sLae[idx] = 2.f * lam * le / (lam + le);
    }
    if (j + 1 < H + TY + 4) {
      const int gn = gy + 1 < ny ? gy + 1 : ny - 1;
      const float ln = !INT && g.solid_row(gn) ? wall_lam(gn) : sRho[idx + FW] * cvk;
      sLan[idx] = 2.f * lam * ln / (lam + ln);
    }
    if (j < H - 3 || j >= H + TY + 3) continue;
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
                      ((sUx[jn * FW + i + 1] - sUx[js * FW + i - 1]) + (sUx[js * FW + i + 1] - sUx[jn * FW + i - 1])) *
                          (1.f / 12.f);
    const float duy = (sUy[jn * FW + i] - sUy[js * FW + i]) * (1.f / 3.f) +
                      ((sUy[jn * FW + i + 1] - sUy[js * FW + i - 1]) + (sUy[jn * FW + i - 1] - sUy[js * FW + i + 1])) *
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
  if (ISO) {
    // Eq. (21): grad(lambda) . grad(T) / (rho cv) joins the advection term as
    // u - grad(lambda) / (rho cv) (u = 0 in solid rows); lambda from rho (ring 5)
#pragma unroll
    for (int m = 0; m < NJ; ++m) {
      const int j = jp + NPH * m;
      const int gy = y0 - H + j;
      if (j < H - 3 || j >= H + TY + 3 || gy < 0 || gy >= ny || g.dirichlet_row(gy)) continue;
      const int idx = j * FW + i;
      const int gs = gy - 1, gn = gy + 1 < ny ? gy + 1 : ny - 1;
      auto lam_at = [&](int row, int jj, int di) -> float {
        return g.solid_row(row) ? wall_lam(row) : sRho[jj * FW + i + di] * cvk;
      };
      const float lE = lam_at(gy, j, 1), lW = lam_at(gy, j, -1);
      const float lN = lam_at(gn, j + 1, 0), lS = lam_at(gs, j - 1, 0);
      const float lNE = lam_at(gn, j + 1, 1), lNW = lam_at(gn, j + 1, -1);
      const float lSE = lam_at(gs, j - 1, 1), lSW = lam_at(gs, j - 1, -1);
      const float glx = (lE - lW) * (1.f / 3.f) + ((lNE - lSW) + (lSE - lNW)) * (1.f / 12.f);
      const float gly = (lN - lS) * (1.f / 3.f) + ((lNE - lSW) + (lNW - lSE)) * (1.f / 12.f);
      const float ircv = sIrcv[idx];
      const float ux = sUx[idx], uy = sUy[idx];
      sUx[idx] = ux - ircv * glx;
      sUy[idx] = uy - ircv * gly;
    }
    __syncthreads();
  }

  // ---- RK4 stages (Eq. 18): stage k on ring 4-k (stage 4 on the output cells
  // only); h1 + 2 h2 + 2 h3 kept in registers
  const float dt = A.dt;
  float acc[NJ];
#pragma unroll
  for (int m = 0; m < NJ; ++m) acc[m] = 0.f;
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    const float* Tc = k == 1 ? sT0 : (k == 3 ? sTb : sTa);
    float* Tn = k == 1 ? sTa : (k == 2 ? sTb : sTa);
    const float cnext = k == 3 ? dt : 0.5f * dt;
    const float wk = (k == 1 || k == 4) ? dt * (1.f / 6.f) : dt * (2.f / 6.f);
    const float wacc = (k == 1) ? 1.f : 2.f;
    const int r = 4 - k;
    // (tested per row rather than through the row flags: these tests use only
    // warp-uniform values and keep the stages within the register budget)
#pragma unroll
    for (int m = 0; m < NJ; ++m) {
      const int j = jp + NPH * m;
      const int gy = y0 - H + j;
      // rows outside ring r are skipped (warp-uniform); every column of a row
      // is evaluated (columns outside the ring are never read later), and only
      // the tile's own cells store or accumulate
      if (j < H - r || j >= H + TY + r || (!INT && (gy < 0 || gy >= ny))) continue;
      const bool own = own_col && j >= H && j < H + TY;
      const int idx = j * FW + i;
      const int js = j - 1, jn = j + 1;
      const float Tp = Tc[idx];
      float hk = 0.f;
      // row 0 under an imposed flux (Section 3.3): beyond the lattice T is the
      // edge copy, and the heat q_in enters through the bottom face instead
      const bool bot = !INT && gy == 0;
      if (ISO && !g.dirichlet_row(gy)) {
        const float TE = Tc[idx + 1], TW = Tc[idx - 1], TN = Tc[jn * FW + i];
        const float TS = bot ? Tp : Tc[js * FW + i];
        const float TNE = Tc[jn * FW + i + 1], TNW = Tc[jn * FW + i - 1];
        const float TSE = bot ? TE : Tc[js * FW + i + 1], TSW = bot ? TW : Tc[js * FW + i - 1];
        // Eq. (20) Laplacian times lambda / (rho cv); the grad(lambda) part of
        // Eq. (21) rides in the advection velocity (after pass C)
        const float lap = (((TNE + TNW) + (TSE + TSW)) + 4.f * ((TE + TW) + (TN + TS)) - 20.f * Tp) * (1.f / 6.f);
        const bool solid = g.solid_row(gy);
        float kk = (solid ? A.kd_w : A.kd) * lap;
        const float gxT = (TE - TW) * (1.f / 3.f) + ((TNE - TSW) + (TSE - TNW)) * (1.f / 12.f);
        const float gyT = (TN - TS) * (1.f / 3.f) + ((TNE - TSW) + (TNW - TSE)) * (1.f / 12.f);
        kk -= sUx[idx] * gxT + sUy[idx] * gyT;
        if (!solid) {
          const float sTr = sqrtf(fmaxf(Tp, 0.f) * A.invTc);
          kk -= sAs[idx] * Tp + sBs[idx] * (1.f + A.kappa * (1.f - sTr)) * sTr;
        }
        if (bot) kk += A.q_in * sIrcv[idx];
        hk = kk;
      } else if (!ISO && (INT || !g.dirichlet_row(gy))) {
        const float TE = Tc[idx + 1], TW = Tc[idx - 1], TN = Tc[jn * FW + i], TS = Tc[js * FW + i];
        // Eqs. (22)-(26): sum of face fluxes over the control volume
        // (an explicit multiply-add chain, so that every kernel that inlines this
        // tile step rounds the face sum the same way)
        float kk = sLae[idx] * (TE - Tp);
        kk = fmaf(sLae[idx - 1], TW - Tp, kk);
        kk = fmaf(sLan[idx], TN - Tp, kk);
        kk = bot ? kk + A.q_in : fmaf(sLan[js * FW + i], TS - Tp, kk);
        kk *= sIrcv[idx];
        if (INT || !g.solid_row(gy)) {
          const float TNE = Tc[jn * FW + i + 1], TNW = Tc[jn * FW + i - 1];
          const float TSE = Tc[js * FW + i + 1], TSW = Tc[js * FW + i - 1];
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
        auto qadd = [&](int q, float x) {
          float h = s_q[q][0][i], l = s_q[q][1][i];
          ff_add(h, l, x);
          s_q[q][0][i] = h;
          s_q[q][1][i] = l;
        };
        if (!INT && gy == 1) qadd(0, wk * sLan[js * FW + i] * (Tc[js * FW + i] - Tp));
        if (!INT && g.top_wall && gy == ny - 2) qadd(1, wk * sLan[idx] * (Tp - Tc[jn * FW + i]));
        if (!INT && gy == A.W) qadd(2, wk * sLan[js * FW + i] * (Tc[js * FW + i] - Tp));
        if (k == 4) {
          const float Tnew = sT0[idx] + dt * (1.f / 6.f) * (acc[m] + hk);
          if (nonfinite(Tnew)) err |= ERR_NONFINITE;
          A.T_out[gy * nx + gx] = Tnew;
          ff_add(ah[P_ENERGY], al[P_ENERGY], Tnew / sIrcv[idx]);
        }
      }
      if (k < 4) Tn[idx] = sT0[idx] + cnext * hk;
    }
    __syncthreads();
    if (k < 4 && has_ghost) {
      fill_ghost(Tn);
      __syncthreads();
    }
  }

  // ---- per-block partials: compensated FP32 through warp and block, FP64 at the end
  warp_flush(P_ENERGY);
  // the wall-flux column partials enter through the first row phase's lanes
  // (the stages' last barrier orders their smem updates before these reads)
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    ah[P_QB + q] = jp == 0 ? s_q[q][0][i] : 0.f;
    al[P_QB + q] = jp == 0 ? s_q[q][1][i] : 0.f;
  }
  warp_flush(P_QB);
  warp_flush(P_QT);
  warp_flush(P_QI);
  if (err) atomicOr(&s_err, err);
  __syncthreads();
  if (tid < NPART) {
    float hi = s_red[0][tid][0], lo = s_red[0][tid][1];
#pragma unroll
    for (int wgi = 1; wgi < NTHREADS / 32; ++wgi) ff_merge(hi, lo, s_red[wgi][tid][0], s_red[wgi][tid][1]);
    A.partials[(long long)part * NPART + tid] = (double)hi + (double)lo;
  }
  if (tid == 0 && s_err) atomicOr(&A.state->error_flags, s_err);
}

// A tile whose frame rows [y0 - HALO, y0 + TY + HALO) all lie in [W + 1, ny - 3]:
// no row of the frame is solid, next to a solid row, the open top row or the
// row below it, so every pull is plain streaming and no wall flux or
// diagnostic row falls in the tile.
__device__ __forceinline__ bool tile_interior(const StepArgs& A, int y0, int TY) {
  return y0 - HALO >= A.W + 1 && y0 + TY + HALO - 1 <= A.ny - 3;
}

template <int TY, int NTH, int MINB>
__global__ void __launch_bounds__(NTH, MINB) k_step(const StepArgs A) {
  extern __shared__ float sm[];
  const float Uc = (float)A.state->Uc, rho_ave = (float)A.state->rho_ave;
  const int part = blockIdx.y * gridDim.x + blockIdx.x;
  if (A.iso)
    step_tile<TY, NTH, false, true>(A, blockIdx.x, blockIdx.y, part, sm, Uc, rho_ave);
  else if (tile_interior(A, blockIdx.y * TY, TY))
    step_tile<TY, NTH, true>(A, blockIdx.x, blockIdx.y, part, sm, Uc, rho_ave);
  else
    step_tile<TY, NTH, false>(A, blockIdx.x, blockIdx.y, part, sm, Uc, rho_ave);
}

// Batched step: the blocks of one launch cover the tiles of every domain of a
// sweep.  blk[b] = (domain, tile within the domain) of block b; the block takes
// that domain's geometry and buffers from the descriptor table, its lagged
// scalars from lag[d] (U/(1+U), mean density) and the shared model parameters
// from its by-value argument (constant bank), and runs the same tile step.
// Stopped domains are skipped.  Two dependent rounds of small loads precede
// the tile.
template <int TY, int NTH, int MINB>
__global__ void __launch_bounds__(NTH, MINB) k_step_batch(const StepArgs P, const DomArgs* __restrict__ desc,
                                                          const int2* __restrict__ blk,
                                                          const int* __restrict__ active,
                                                          const float2* __restrict__ lag) {
  extern __shared__ float sm[];
  __shared__ DomArgs sD;
  __shared__ int s_act;
  __shared__ int2 s_bl;
  __shared__ float2 s_lg;
  {
    const int2 bl = blk[blockIdx.x];
    const int* src = reinterpret_cast<const int*>(desc + bl.x);
    int* dst = reinterpret_cast<int*>(&sD);
    for (int q = threadIdx.x; q < (int)(sizeof(DomArgs) / sizeof(int)); q += NTH) dst[q] = src[q];
    if (threadIdx.x == NTH - 1) {
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
  const int local = s_bl.y;
  const int tx = (A.nx + TILE_W - 1) / TILE_W;
  const int by = local / tx;
  if (tile_interior(A, by * TY, TY))
    step_tile<TY, NTH, true>(A, local % tx, by, local, sm, s_lg.x, s_lg.y);
  else
    step_tile<TY, NTH, false>(A, local % tx, by, local, sm, s_lg.x, s_lg.y);
}

// The lagged scalars of a domain as the batched step reads them.
__global__ void k_lag_from_state(const DevState* st, float2* lag) {
  if (threadIdx.x == 0) *lag = make_float2((float)st->Uc, (float)st->rho_ave);
}

// FP64 reduction of the per-block partials (one CTA); updates the lagged
// scalars of the next step and the diagnostics record.
__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ partials, int nblk, DevState* st,
                                                 double inv_nfluid, double inv_nx, double* hist, int hist_cap) {
  __shared__ double s_red[8][NPART];
  double v[NPART];
#pragma unroll
  for (int q = 0; q < NPART; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NPART; ++q) v[q] += partials[(long long)b * NPART + q];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NPART; ++q) {
    const double s = warp_sum(v[q]);
    if (lane == 0) s_red[warp][q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[NPART];
#pragma unroll
    for (int q = 0; q < NPART; ++q) {
      s[q] = 0.0;
      for (int wgi = 0; wgi < 8; ++wgi) s[q] += s_red[wgi][q];
    }
    st->rho_ave_prev = st->rho_ave;
    st->rho_ave = s[P_MASS] * inv_nfluid;
    const double ut = s[P_UTOP] * inv_nx;
    st->u_top = ut;
    st->U = ut > 0.0 ? ut : 0.0;
    st->Uc = st->U / (1.0 + st->U);
    st->step += 1;
    st->mass = s[P_MASS];
    st->energy = s[P_ENERGY];
    st->q_bottom = s[P_QB] * inv_nx;
    st->q_top = s[P_QT] * inv_nx;
    st->q_interface = s[P_QI] * inv_nx;
    st->q_sum += st->q_bottom;
    st->q_count += 1;
    st->vcov = s[P_VCOV] * inv_nx;
    st->vcov_sum += st->vcov;
    if (hist && st->hist_len < hist_cap) hist[st->hist_len++] = st->q_bottom;
  }
}

// One CTA per domain of a batch: the same reduction as k_reduce.
struct ReduceArgs {
  const double* partials;
  DevState* state;
  double* hist;
  int nblk;
  double inv_nfluid, inv_nx;
};

__global__ void __launch_bounds__(256) k_reduce_batch(const ReduceArgs* __restrict__ ra,
                                                       const int* __restrict__ active, float2* lag, int hist_cap) {
  const int d = blockIdx.x;
  if (!active[d]) return;
  const ReduceArgs r = ra[d];
  __shared__ double s_red[8][NPART];
  double v[NPART];
#pragma unroll
  for (int q = 0; q < NPART; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < r.nblk; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NPART; ++q) v[q] += r.partials[(long long)b * NPART + q];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NPART; ++q) {
    const double s = warp_sum(v[q]);
    if (lane == 0) s_red[warp][q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[NPART];
#pragma unroll
    for (int q = 0; q < NPART; ++q) {
      s[q] = 0.0;
      for (int wgi = 0; wgi < 8; ++wgi) s[q] += s_red[wgi][q];
    }
    DevState* st = r.state;
    st->rho_ave_prev = st->rho_ave;
    st->rho_ave = s[P_MASS] * r.inv_nfluid;
    const double ut = s[P_UTOP] * r.inv_nx;
    st->u_top = ut;
    st->U = ut > 0.0 ? ut : 0.0;
    st->Uc = st->U / (1.0 + st->U);
    st->step += 1;
    st->mass = s[P_MASS];
    st->energy = s[P_ENERGY];
    st->q_bottom = s[P_QB] * r.inv_nx;
    st->q_top = s[P_QT] * r.inv_nx;
    st->q_interface = s[P_QI] * r.inv_nx;
    st->q_sum += st->q_bottom;
    st->q_count += 1;
    st->vcov = s[P_VCOV] * r.inv_nx;
    st->vcov_sum += st->vcov;
    if (r.hist && st->hist_len < hist_cap) r.hist[st->hist_len++] = st->q_bottom;
    lag[d] = make_float2((float)st->Uc, (float)st->rho_ave);
  }
}

// Initial state: f* = rest equilibrium w_i rho (deviation form), T with the
// Dirichlet rows set, the convective-outlet memory, and per-block fluid mass.
__global__ void __launch_bounds__(256) k_init(const StepArgs A, const float* __restrict__ rho0,
                                              const float* __restrict__ T0, float* __restrict__ f,
                                              float* __restrict__ T, float* __restrict__ ftop_a,
                                              float* __restrict__ ftop_b) {
  const Geo g = make_geo(A);
  const long long N = A.plane;  // population plane stride (>= nx ny)
  const long long NC = (long long)A.nx * A.ny;
  double mass = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < NC; c += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(c / A.nx), x = (int)(c % A.nx);
    const bool solid = g.solid_row(y);
    const float d = solid ? 0.f : rho0[c] - A.rho_ref;
    const float w[9] = {4.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f,
                        1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};
#pragma unroll
    for (int q = 0; q < 9; ++q) f[q * N + c] = solid ? 0.f : w[q] * d;
    T[c] = g.dirichlet_row(y) ? (y == 0 ? A.T_bottom : A.T_top) : T0[c];
    if (!solid) mass += (double)rho0[c];
    if (y == A.ny - 1 && ftop_a) {
      ftop_a[x] = w[4] * d;
      ftop_a[A.nx + x] = w[7] * d;
      ftop_a[2 * A.nx + x] = w[8] * d;
      ftop_b[x] = w[4] * d;
      ftop_b[A.nx + x] = w[7] * d;
      ftop_b[2 * A.nx + x] = w[8] * d;
    }
  }
  __shared__ double s_red[8];
  const double s = warp_sum(mass);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += s_red[q];
    A.partials[(long long)blockIdx.x * NPART + P_MASS] = t;
  }
}

__global__ void k_init_state(const double* __restrict__ partials, int nblk, DevState* st, double inv_nfluid) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double m = 0.0;
    for (int b = 0; b < nblk; ++b) m += partials[(long long)b * NPART + P_MASS];
    st->rho_ave = m * inv_nfluid;
    st->rho_ave_prev = st->rho_ave;
    st->U = 0.0;
    st->Uc = 0.0;
    st->step = 0;
    st->mass = m;
    st->energy = 0.0;
    st->q_bottom = st->q_top = st->q_interface = st->u_top = 0.0;
    st->q_sum = 0.0;
    st->q_count = 0;
    st->vcov = st->vcov_sum = 0.0;
    st->error_flags = 0;
    st->hist_len = 0;
  }
}

// rho^n and u^n from the stored post-collision populations: collision keeps
// mass and leaves sum_i e_i f*_i = rho u + F/2 (Eqs. 2, 5, 8), so
// u = (sum e f* - F/2) / rho with F recomputed from rho^n and T^n.
__global__ void __launch_bounds__(256) k_read(const StepArgs A, const float* __restrict__ Tn, int zero_u,
                                              float* rho_out, float* ux_out, float* uy_out) {
  const Geo g = make_geo(A);
  const long long N = A.plane;  // population plane stride (>= nx ny)
  const long long NC = (long long)A.nx * A.ny;
  const float rho_ave = (float)A.state->rho_ave_prev;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < NC; c += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(c / A.nx), x = (int)(c % A.nx);
    if (g.solid_row(y)) {
      if (rho_out) rho_out[c] = 0.f;
      if (ux_out) ux_out[c] = 0.f;
      if (uy_out) uy_out[c] = 0.f;
      continue;
    }
    float psi_nb[3][3];
    float rho = 0.f, jx = 0.f, jy = 0.f;
    for (int dy = -1; dy <= 1; ++dy) {
      int yy = y + dy;
      yy = yy > A.ny - 1 ? A.ny - 1 : yy;  // zero-gradient ghost above an open top
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = wrapx(x + dx, A.nx);
        float ps = 0.f;
        if (!g.solid_row(yy)) {
          const long long o = (long long)yy * A.nx + xx;
          float f[9];
#pragma unroll
          for (int q = 0; q < 9; ++q) f[q] = A.f_out[q * N + o];
          const float r = A.rho_ref + sum9(f);
          const float T = A.eos_T_fixed ? A.Ts : Tn[o];
          ps = sqrtf(fmaxf(pr_psi2(A, r, T), 0.f));
          if (dx == 0 && dy == 0) {
            rho = r;
            jx = (f[1] - f[3]) + ((f[5] - f[6]) - (f[7] - f[8]));
            jy = (f[2] - f[4]) + ((f[5] + f[6]) - (f[7] + f[8]));
          }
        }
        psi_nb[dy + 1][dx + 1] = ps;
      }
    }
    const float psi = psi_nb[1][1];
    const bool sol_s = g.solid_row(y - 1);
    const bool sol_n = g.solid_row(y + 1 > A.ny - 1 ? A.ny - 1 : y + 1);
    for (int dx = 0; dx < 3; ++dx) {
      if (sol_s) psi_nb[0][dx] = psi;
      if (sol_n) psi_nb[2][dx] = psi;
    }
    const float sx = (psi_nb[1][2] - psi_nb[1][0]) * (1.f / 3.f) +
                     ((psi_nb[2][2] - psi_nb[2][0]) + (psi_nb[0][2] - psi_nb[0][0])) * (1.f / 12.f);
    const float sy = (psi_nb[2][1] - psi_nb[0][1]) * (1.f / 3.f) +
                     ((psi_nb[2][2] + psi_nb[2][0]) - (psi_nb[0][2] + psi_nb[0][0])) * (1.f / 12.f);
    const float Fx = -A.G * psi * sx;
    const float Fy = -A.G * psi * sy + A.Gw[x] * psi * psi * ((float)sol_n - (float)sol_s) * (1.f / 6.f) +
                     (rho - rho_ave) * A.g_y;
    if (rho_out) rho_out[c] = rho;
    if (ux_out) ux_out[c] = zero_u ? 0.f : (jx - 0.5f * Fx) / rho;
    if (uy_out) uy_out[c] = zero_u ? 0.f : (jy - 0.5f * Fy) / rho;
  }
}

}  // namespace hlb
