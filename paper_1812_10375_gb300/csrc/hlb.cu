// Host side of the C ABI declared in include/hlb.h: parameter handling, the
// Peng-Robinson coexistence solver, workspace layout, kernel launches and
// CUDA-graph replay of the step.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "hlb.h"
#include "hlb_kernels.cuh"
#include "hlb_march.cuh"
#include "hlb_split.cuh"
#include "hlb_energy_walk.cuh"
#include "hlb_substep.cuh"

using namespace hlb;

namespace {

constexpr int TILE_X = TILE_W;  // 52 output columns in a 64-wide frame

// Compiled variants of the fused step kernel (tile height, threads per CTA).
struct Variant {
  int ty, nth;
  size_t smem;
  const void* single_fn;
  const void* batch_fn;
  void (*launch_single)(dim3, size_t, cudaStream_t, const StepArgs&);
  void (*launch_batch)(int, size_t, cudaStream_t, const StepArgs&, const DomArgs*, const int2*, const int*,
                       const float2*);
};

template <int TY, int NTH, int MINB>
void launch_single_v(dim3 grid, size_t smem, cudaStream_t s, const StepArgs& a) {
  k_step<TY, NTH, MINB><<<grid, NTH, smem, s>>>(a);
}
template <int TY, int NTH, int MINB>
void launch_batch_v(int blocks, size_t smem, cudaStream_t s, const StepArgs& phys, const DomArgs* desc,
                    const int2* blk, const int* act, const float2* lag) {
  k_step_batch<TY, NTH, MINB><<<blocks, NTH, smem, s>>>(phys, desc, blk, act, lag);
}

#define HLB_VARIANT_ENTRY(TY, NTH, MINB)                                                              \
  Variant{TY, NTH, (size_t)step_smem_floats<TY>() * sizeof(float), (const void*)k_step<TY, NTH, MINB>, \
          (const void*)k_step_batch<TY, NTH, MINB>, launch_single_v<TY, NTH, MINB>,                   \
          launch_batch_v<TY, NTH, MINB>},
const Variant VARIANTS[] = {HLB_STEP_VARIANTS(HLB_VARIANT_ENTRY)};
constexpr int NVARIANTS = (int)(sizeof(VARIANTS) / sizeof(VARIANTS[0]));
constexpr int TILE_Y = 28;      // the default variant's tile height (variant 0)
constexpr int MIN_TILE_Y = 16;  // the shortest variant tile (sizes the partial-sum slots)

// Split-step variants (k_flow* then k_energy*): the flow tile's fluid rows and
// threads, and the energy kernel's thread layout (the energy tile is the same).
struct FlowVariant {
  int ty, nth;
  int ewalk;   // energy kernel: 0 tile, 1 row walk
  int ep;      // energy tile: rows per run; walk: segment rows
  size_t smem;
  const void* single_fn;
  const void* batch_fn;
  const void* esingle_fn;
  const void* ebatch_fn;
  size_t esmem;  // dynamic shared memory of the energy kernels
  void (*launch_single)(dim3, size_t, cudaStream_t, const StepArgs&);
  void (*launch_batch)(int, size_t, cudaStream_t, const StepArgs&, const DomArgs*, const int2*, const int*,
                       const float2*);
  void (*energy_single)(dim3, cudaStream_t, const StepArgs&, int, int);
  void (*energy_batch)(int, cudaStream_t, const StepArgs&, const DomArgs*, const int2*, const int*, int, int);
  dim3 egrid(int nx, int ny) const {
    return ewalk ? dim3((nx + EW_OUT - 1) / EW_OUT, (ny + ep - 1) / ep) : dim3((nx + EN_TX - 1) / EN_TX, (ny + EN_TY - 1) / EN_TY);
  }
};
template <int TY, int NTH, int MINB, bool RP>
void launch_flow_single(dim3 grid, size_t smem, cudaStream_t s, const StepArgs& a) {
  k_flow<TY, NTH, MINB, RP><<<grid, NTH, smem, s>>>(a);
}
template <int TY, int NTH, int MINB, bool RP>
void launch_flow_batch(int blocks, size_t smem, cudaStream_t s, const StepArgs& phys, const DomArgs* desc,
                       const int2* blk, const int* act, const float2* lag) {
  k_flow_batch<TY, NTH, MINB, RP><<<blocks, NTH, smem, s>>>(phys, desc, blk, act, lag);
}
template <int R, int NPH, int MINB>
void launch_energy_single(dim3 grid, cudaStream_t s, const StepArgs& a, int sub, int nsub) {
  k_energy<R, NPH, MINB><<<grid, 64 * NPH, energy_smem_bytes(), s>>>(a, sub, nsub);
}
template <int R, int NPH, int MINB>
void launch_energy_batch(int blocks, cudaStream_t s, const StepArgs& phys, const DomArgs* desc, const int2* blk,
                         const int* act, int sub, int nsub) {
  k_energy_batch<R, NPH, MINB><<<blocks, 64 * NPH, energy_smem_bytes(), s>>>(phys, desc, blk, act, sub, nsub);
}
template <int L, int MINB, int PF>
void launch_walk_single(dim3 grid, cudaStream_t s, const StepArgs& a, int sub, int nsub) {
  k_energy_walk<L, MINB, PF><<<grid, EW_W, 0, s>>>(a, sub, nsub);
}
template <int L, int MINB, int PF>
void launch_walk_batch(int blocks, cudaStream_t s, const StepArgs& phys, const DomArgs* desc, const int2* blk,
                       const int* act, int sub, int nsub) {
  k_energy_walk_batch<L, MINB, PF><<<blocks, EW_W, 0, s>>>(phys, desc, blk, act, sub, nsub);
}
#define HLB_SPLIT_TILE(TY, NTH, MINB, RP, ER, ENPH, EMINB)                                                      \
  FlowVariant{TY, NTH, 0, ER, flow_smem_bytes<TY>(), (const void*)k_flow<TY, NTH, MINB, RP>,                    \
              (const void*)k_flow_batch<TY, NTH, MINB, RP>, (const void*)k_energy<ER, ENPH, EMINB>,           \
              (const void*)k_energy_batch<ER, ENPH, EMINB>, energy_smem_bytes(),                              \
              launch_flow_single<TY, NTH, MINB, RP>, launch_flow_batch<TY, NTH, MINB, RP>,                    \
              launch_energy_single<ER, ENPH, EMINB>, launch_energy_batch<ER, ENPH, EMINB>},
#define HLB_SPLIT_WALK(TY, NTH, MINB, RP, L, EMINB, PF)                                                         \
  FlowVariant{TY, NTH, 1, L, flow_smem_bytes<TY>(), (const void*)k_flow<TY, NTH, MINB, RP>,                     \
              (const void*)k_flow_batch<TY, NTH, MINB, RP>, (const void*)k_energy_walk<L, EMINB, PF>,         \
              (const void*)k_energy_walk_batch<L, EMINB, PF>, 0, launch_flow_single<TY, NTH, MINB, RP>,       \
              launch_flow_batch<TY, NTH, MINB, RP>, launch_walk_single<L, EMINB, PF>,                         \
              launch_walk_batch<L, EMINB, PF>},
const FlowVariant FLOWS[] = {HLB_SPLIT_VARIANTS(HLB_SPLIT_TILE, HLB_SPLIT_WALK)};
constexpr int NSPLIT = (int)(sizeof(FLOWS) / sizeof(FLOWS[0]));
constexpr int MIN_FLOW_TY = 8;  // the shortest flow tile (sizes the flow partial-sum slots)

// Variant numbering: [0, NSPLIT) split step, then the fused tiled kernels
// (VARIANTS), then the row-marching kernels (k_march*: segments of
// MARCH_SEGS[k] rows with one thread per column; only for nx <= MARCH_MAX_NX).
#define HLB_MARCH_ENTRY(S) S,
constexpr int MARCH_SEGS[] = {HLB_MARCH_SEGMENTS(HLB_MARCH_ENTRY)};
constexpr int NMARCH = (int)(sizeof(MARCH_SEGS) / sizeof(MARCH_SEGS[0]));
constexpr int NV_ALL = NSPLIT + NVARIANTS + NMARCH;
constexpr int FIRST_TILED = NSPLIT;
static_assert(MARCH_SEGS[0] >= MIN_TILE_Y, "march segments must not outnumber the partial-sum slots");
bool is_split(int v) { return v < NSPLIT; }
bool is_march(int v) { return v >= NSPLIT + NVARIANTS; }
int tiled_index(int v) { return v - NSPLIT; }  // index into VARIANTS of a fused tiled variant
int march_seg(int v) { return MARCH_SEGS[v - NSPLIT - NVARIANTS]; }
size_t march_smem(int nx) { return (size_t)march_smem_floats(nx) * sizeof(float); }

int fluid_rows_of(int ny, int W, int top_bc) { return fluid_end(ny, top_bc) - W; }

// Launch grid of the step kernel of variant v (the flow kernel for a split variant).
dim3 grid_of(int nx, int ny, int W, int top_bc, int v) {
  if (is_split(v)) {
    const int ty = FLOWS[v].ty;
    return dim3((nx + FL_TX - 1) / FL_TX, (fluid_rows_of(ny, W, top_bc) + ty - 1) / ty);
  }
  if (is_march(v)) return dim3((ny + march_seg(v) - 1) / march_seg(v), 1);
  const int t = tiled_index(v);
  return dim3((nx + TILE_X - 1) / TILE_X, (ny + VARIANTS[t].ty - 1) / VARIANTS[t].ty);
}
// The largest energy grid of any split variant (sizes the energy partial-sum slots).
dim3 energy_grid_of(int nx, int ny) { return dim3((nx + EN_TX - 1) / EN_TX, (ny + EN_TY - 1) / EN_TY); }
static_assert(EW_OUT == EN_TX, "walk strips and energy tiles share the column split");
size_t flow_part_slots(int nx, int ny, int W, int top_bc) {
  return (size_t)((nx + FL_TX - 1) / FL_TX) * ((fluid_rows_of(ny, W, top_bc) + MIN_FLOW_TY - 1) / MIN_FLOW_TY);
}
constexpr int GRAPH_STEPS = 16;     // steps per captured graph (even: buffers return to parity 0)
constexpr int HIST_CAP = 1 << 16;   // wall-flux history entries kept per domain
constexpr int INIT_BLOCKS = 304;
constexpr int MAX_SUB = 64;  // largest N of Eq. (27)

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// ------------------------------------------------------------ Peng-Robinson
// Eq. (28) written in the specific volume v = 1/rho:
//   p = R T / (v - b) - a phi(T) / (v^2 + 2 b v - b^2)
// whose antiderivative in v is
//   Pi(v) = R T ln(v - b) - a phi / (2 sqrt2 b) ln((v + b - sqrt2 b) / (v + b + sqrt2 b)).
struct PRHost {
  double a, b, R, kappa, Tc;
  double alpha(double T) const { return 1.0 + kappa * (1.0 - sqrt(fmax(T, 0.0) / Tc)); }
  double phi(double T) const { double al = alpha(T); return al * al; }
  double p_rho(double rho, double T) const {
    return rho * R * T / (1.0 - b * rho) - a * phi(T) * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
  }
  double dp_drho(double rho, double T) const {
    const double den = 1.0 + 2.0 * b * rho - b * b * rho * rho;
    const double dden = 2.0 * b - 2.0 * b * b * rho;
    return R * T / ((1.0 - b * rho) * (1.0 - b * rho)) - a * phi(T) * (2.0 * rho * den - rho * rho * dden) / (den * den);
  }
  double log_term(double v) const {
    const double s2b = sqrt(2.0) * b;
    return log((v + b - s2b) / (v + b + s2b));
  }
  double Pi(double v, double T) const { return R * T * log(v - b) - a * phi(T) / (2.0 * sqrt(2.0) * b) * log_term(v); }
  // antiderivative of T (dp/dT)_v:  T dphi/dT = -kappa alpha(T) sqrt(T/Tc)
  double Hi(double v, double T) const {
    const double Tdphi = -kappa * alpha(T) * sqrt(fmax(T, 0.0) / Tc);
    return R * T * log(v - b) - a * Tdphi / (2.0 * sqrt(2.0) * b) * log_term(v);
  }
};

template <typename F>
double bisect(F f, double lo, double hi) {
  double flo = f(lo);
  for (int it = 0; it < 400; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    const double fm = f(mid);
    if ((fm < 0) == (flo < 0)) {
      lo = mid;
      flo = fm;
    } else {
      hi = mid;
    }
  }
  return 0.5 * (lo + hi);
}

// Maxwell equal-area construction: p(v_l) = p(v_v) = p_s and
// Pi(v_v) - Pi(v_l) = p_s (v_v - v_l).
bool coexistence(const PRHost& e, double T, double* rl, double* rv, double* hfg) {
  const double rmax = 0.999999 / e.b;
  // spinodals: sign changes of dp/drho on a grid, refined by bisection
  const int NG = 20000;
  double sp[2];
  int ns = 0;
  double prev = e.dp_drho(1e-6, T);
  for (int k = 1; k <= NG && ns < 2; ++k) {
    const double r = 1e-6 + (rmax - 1e-6) * k / NG;
    const double d = e.dp_drho(r, T);
    if ((d < 0) != (prev < 0)) {
      const double r0 = 1e-6 + (rmax - 1e-6) * (k - 1) / NG;
      sp[ns++] = bisect([&](double x) { return e.dp_drho(x, T); }, r0, r);
    }
    prev = d;
  }
  if (ns < 2) return false;
  const double s1 = sp[0], s2 = sp[1];
  const double p_hi = e.p_rho(s1, T);
  const double p_lo = fmax(e.p_rho(s2, T), 1e-14);
  auto roots = [&](double ps, double* v_v, double* v_l) {
    const double r_min = 0.5 * ps / (e.R * T);
    const double rvap = bisect([&](double r) { return e.p_rho(r, T) - ps; }, r_min, s1);
    const double rliq = bisect([&](double r) { return e.p_rho(r, T) - ps; }, s2, rmax);
    *v_v = 1.0 / rvap;
    *v_l = 1.0 / rliq;
  };
  auto area = [&](double ps) {
    double vv, vl;
    roots(ps, &vv, &vl);
    return (e.Pi(vv, T) - e.Pi(vl, T)) - ps * (vv - vl);
  };
  const double eps = 1e-12 * (p_hi - p_lo);
  const double ps = bisect(area, p_lo + eps, p_hi - eps);
  double vv, vl;
  roots(ps, &vv, &vl);
  *rl = 1.0 / vl;
  *rv = 1.0 / vv;
  if (hfg) *hfg = e.Hi(vv, T) - e.Hi(vl, T);  // Eq. (14)
  return true;
}

PRHost pr_of(const hlb_params* p) {
  PRHost e;
  e.a = p->a;
  e.b = p->b;
  e.R = p->R;
  e.kappa = 0.37464 + 1.54226 * p->omega - 0.26992 * p->omega * p->omega;
  e.Tc = (p->a / p->b) * (0.0778 / 0.45724) / p->R;
  return e;
}

// Smallest N of Eq. (27) for which one RK4 sub-step of dt/N is stable for the
// finite-volume conduction operator.  The operator is C^-1 K (C the diagonal
// heat capacities, K symmetric), so its eigenvalues are real and <= 0; by
// Gershgorin they lie in [-2 S, 0] with S the largest sum over a cell's four
// faces of lambda_f / (rho c)_P, and a harmonic face conductivity is at most
// twice the cell's own, so |eigenvalue| <= 16 D_max with D = lambda / (rho c)
// of a material (k in the fluid, lambda_w / (rho_w c_w) in the heater).  RK4's
// stability interval on the negative real axis reaches 2.785.  The advection
// and latent-heat terms are not in the bound: at the method's velocities they
// are small beside it.  0 when the coexistence densities needed for the
// heater's defaults do not exist.
int stable_substeps(const hlb_params* p) {
  double rho_l = p->rho_l;
  if (!(rho_l > 0)) {
    const PRHost e = pr_of(p);
    double rv;
    if (!coexistence(e, p->Ts_over_Tc * e.Tc, &rho_l, &rv, nullptr)) return 0;
  }
  const double rho_w = p->rho_w > 0 ? p->rho_w : 3.0 * rho_l;
  const double cv_w = p->cv_w > 0 ? p->cv_w : p->cv;
  const double lam_w = p->lambda_w > 0 ? p->lambda_w : 3.0 * rho_l * p->cv * p->k;
  const double D = fmax(p->k, lam_w / (rho_w * cv_w));
  const double RK4_REAL_AXIS = 2.785;
  const double n = ceil(16.0 * D / RK4_REAL_AXIS);
  if (!(n < 1e6)) return 0;
  return n < 1.0 ? 1 : (int)n;
}

// N of Eq. (27) a parameter set runs with: n_sub, or the bound above when it is 0.
int resolved_nsub(const hlb_params* p) { return p->n_sub != 0 ? p->n_sub : stable_substeps(p); }

// Stride of the population planes in floats: nx ny rounded up to whole
// 128-byte lines, so that every plane starts on a line.
size_t plane_stride(size_t N) { return (N + 31) / 32 * 32; }

bool params_valid(const hlb_params* p) {
  if (!p) return false;
  if (p->nx < 4 || p->ny < 6 || p->wall_rows < 1) return false;
  if (p->top_bc < HLB_TOP_WALL || p->top_bc > HLB_TOP_CONVECTIVE) return false;
  const int fluid_rows = p->ny - p->wall_rows - (p->top_bc == HLB_TOP_WALL ? 1 : 0);
  if (fluid_rows < 3) return false;
  if (p->n_sub < 0 || p->n_sub > MAX_SUB) return false;
  if (p->storage != HLB_STORE_DEVIATION && p->storage != HLB_STORE_PLAIN) return false;
  if (p->diffusion != HLB_DIFF_FV && p->diffusion != HLB_DIFF_ISO) return false;
  if (p->bottom_bc != HLB_BOTTOM_DIRICHLET && p->bottom_bc != HLB_BOTTOM_FLUX) return false;
  if (!isfinite(p->q_in)) return false;
  if (!(p->a > 0 && p->b > 0 && p->R > 0 && p->Ts_over_Tc > 0)) return false;
  if (!(p->s_e > 0 && p->s_e < 2 && p->s_zeta > 0 && p->s_zeta < 2 && p->s_j > 0 && p->s_j < 2 &&
        p->s_q > 0 && p->s_q < 2))
    return false;
  if (!(p->tau_l > 0.5 && p->tau_v > 0.5 && p->cv > 0 && p->k > 0)) return false;
  // the kernels address a cell's nine populations with 32-bit offsets (q plane + cell)
  if (p->nx > (1 << 20) || p->ny > (1 << 20)) return false;
  if (9 * (long long)plane_stride((size_t)p->nx * p->ny) >= (1LL << 31)) return false;
  // N of Eq. (27): the fused kernel takes the first sub-step, k_energy_substep
  // the others (finite-volume scheme only)
  const int nsub = resolved_nsub(p);
  if (nsub < 1 || nsub > MAX_SUB) return false;
  if (nsub > 1 && p->diffusion != HLB_DIFF_FV) return false;
  return true;
}

}  // namespace

// ------------------------------------------------------------------ handle
struct hlb_domain {
  hlb_params p;
  double Tc = 0, rho_ref = 0;
  cudaStream_t stream = nullptr;
  float* f[2] = {nullptr, nullptr};
  float* T[2] = {nullptr, nullptr};
  float* Gw = nullptr;
  float* ftop[2] = {nullptr, nullptr};
  double* partials = nullptr;
  DevState* state = nullptr;
  double* hist = nullptr;
  // N > 1 (Eq. 27): rho^n, u_x^n, u_y^n of the step, a T buffer and the
  // sub-steps' per-block partials
  float* mom = nullptr;
  float* Tscr = nullptr;
  double* subpart = nullptr;
  dim3 sub_grid;
  // split step: per-tile partials of the flow and energy kernels, energy grid
  double* fpart = nullptr;
  double* epart = nullptr;
  dim3 egrid;
  int parity = 0;
  long long steps = 0;
  bool fields_set = false;
  int host_flags = 0;
  long long n_fluid = 0;
  dim3 grid;
  size_t smem = 0;
  int variant = 0;
  StepArgs base;
  cudaGraphExec_t graph = nullptr;
};

namespace {

// Variant v for domain d: launch grids of its step kernel(s).
void set_variant_grids(hlb_domain* d, int v) {
  d->variant = v;
  d->grid = grid_of(d->p.nx, d->p.ny, d->p.wall_rows, d->p.top_bc, v);
  d->egrid = is_split(v) ? FLOWS[v].egrid(d->p.nx, d->p.ny) : energy_grid_of(d->p.nx, d->p.ny);
}

}  // namespace

namespace {

struct Layout {
  size_t f, T, Gw, ftop, partials, state, hist, mom, fpart, epart, sub, total;
};

dim3 sub_grid_of(int nx, int ny) { return dim3((nx + SUB_TX - 1) / SUB_TX, (ny + SUB_TY - 1) / SUB_TY); }

Layout layout_of(const hlb_params* p) {
  Layout L;
  const size_t N = (size_t)p->nx * p->ny;
  const size_t PS = plane_stride(N);
  const size_t nblk = (size_t)((p->nx + TILE_X - 1) / TILE_X) * ((p->ny + MIN_TILE_Y - 1) / MIN_TILE_Y);
  size_t o = 0;
  L.f = o;        o += align_up(2 * 9 * PS * sizeof(float));
  L.T = o;        o += align_up(2 * N * sizeof(float));
  L.Gw = o;       o += align_up((size_t)p->nx * sizeof(float));
  L.ftop = o;     o += align_up(2 * 3 * (size_t)p->nx * sizeof(float));
  L.partials = o; o += align_up((nblk > INIT_BLOCKS ? nblk : INIT_BLOCKS) * NPART * sizeof(double));
  L.state = o;    o += align_up(sizeof(DevState));
  L.hist = o;     o += align_up(HIST_CAP * sizeof(double));
  // rho^n, u_x^n, u_y^n of the step and a T plane for sub-steps
  L.mom = o;      o += align_up(4 * N * sizeof(float));
  L.fpart = o;    o += align_up(flow_part_slots(p->nx, p->ny, p->wall_rows, p->top_bc) * NFPART * sizeof(double));
  const dim3 eg = energy_grid_of(p->nx, p->ny);
  L.epart = o;    o += align_up((size_t)eg.x * eg.y * NEPART * sizeof(double));
  L.sub = o;
  if (resolved_nsub(p) > 1) {
    // the fused kernels' sub-step partials (Eq. 27)
    const dim3 sg = sub_grid_of(p->nx, p->ny);
    o += align_up((size_t)sg.x * sg.y * NSUBPART * sizeof(double));
  }
  L.total = o;
  return L;
}

size_t smem_bytes() {
  return VARIANTS[0].smem;
}

StepArgs args_for(hlb_domain* d, int par) {
  StepArgs a = d->base;
  a.f_in = d->f[par];
  a.f_out = d->f[par ^ 1];
  a.T_in = d->T[par];
  a.T_out = d->T[par ^ 1];
  a.ftop_in = d->ftop[par];
  a.ftop_out = d->ftop[par ^ 1];
  return a;
}

// One step of the split form: the flow kernel, N energy sub-steps, the reduction.
hlb_status launch_split_step(hlb_domain* d, cudaEvent_t after_flow = nullptr, cudaEvent_t after_energy = nullptr) {
  const StepArgs a = args_for(d, d->parity);
  const FlowVariant& fv = FLOWS[d->variant];
  fv.launch_single(d->grid, fv.smem, d->stream, a);
  if (after_flow && cudaEventRecord(after_flow, d->stream) != cudaSuccess) return HLB_ECUDA;
  const int nsub = d->p.n_sub;
  for (int s = 1; s <= nsub; ++s) fv.energy_single(d->egrid, d->stream, a, s, nsub);
  if (after_energy && cudaEventRecord(after_energy, d->stream) != cudaSuccess) return HLB_ECUDA;
  k_reduce_split<<<1, 256, 0, d->stream>>>(d->fpart, (int)(d->grid.x * d->grid.y), d->epart,
                                           (int)(d->egrid.x * d->egrid.y), d->state, 1.0 / (double)d->n_fluid,
                                           1.0 / (double)d->p.nx, d->hist, HIST_CAP);
  if (cudaGetLastError() != cudaSuccess) return HLB_ECUDA;
  d->parity ^= 1;
  d->steps += 1;
  return HLB_OK;
}

hlb_status launch_step(hlb_domain* d) {
  if (is_split(d->variant)) return launch_split_step(d);
  const StepArgs a = args_for(d, d->parity);
  if (is_march(d->variant)) {
    k_march<<<d->grid, march_row_stride(d->p.nx), march_smem(d->p.nx), d->stream>>>(a, march_seg(d->variant));
  } else {
    const Variant& tv = VARIANTS[tiled_index(d->variant)];
    tv.launch_single(d->grid, tv.smem, d->stream, a);
  }
  k_reduce<<<1, 256, 0, d->stream>>>(d->partials, (int)(d->grid.x * d->grid.y), d->state, 1.0 / (double)d->n_fluid,
                                     1.0 / (double)d->p.nx, d->hist, HIST_CAP);
  if (d->p.n_sub > 1) {
    // Eq. (27): sub-steps 2..N on the step's rho^n and u^n (recovered from the
    // post-collision populations and T^n, with the mean density the step used)
    const size_t N = (size_t)d->p.nx * d->p.ny;
    float* rho = d->mom;
    float* ux = d->mom + N;
    float* uy = d->mom + 2 * N;
    k_read<<<INIT_BLOCKS, 256, 0, d->stream>>>(a, d->T[d->parity], 0, rho, ux, uy);
    float* Tcur = d->T[d->parity ^ 1];
    float* Tother = d->Tscr;
    const int nsub = d->p.n_sub;
    for (int s = 2; s <= nsub; ++s) {
      k_energy_substep<<<d->sub_grid, SUB_NT, sub_smem_bytes(), d->stream>>>(a, rho, ux, uy, Tcur, Tother,
                                                                             d->subpart, s == 2, s == nsub);
      float* t = Tcur;
      Tcur = Tother;
      Tother = t;
    }
    if (Tcur != d->T[d->parity ^ 1] &&
        cudaMemcpyAsync(d->T[d->parity ^ 1], Tcur, N * sizeof(float), cudaMemcpyDeviceToDevice, d->stream) !=
            cudaSuccess)
      return HLB_ECUDA;
    k_substep_fix<<<1, 256, 0, d->stream>>>(d->subpart, (int)(d->sub_grid.x * d->sub_grid.y), d->state,
                                            1.0 / (double)d->p.nx, d->hist);
  }
  if (cudaGetLastError() != cudaSuccess) return HLB_ECUDA;
  d->parity ^= 1;
  d->steps += 1;
  return HLB_OK;
}

void drop_graph(hlb_domain* d) {
  if (d->graph) {
    cudaGraphExecDestroy(d->graph);
    d->graph = nullptr;
  }
}

hlb_status build_graph(hlb_domain* d) {
  // capture GRAPH_STEPS steps starting from parity 0
  if (d->parity != 0) return HLB_ESTATE;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HLB_ECUDA;
  const long long s0 = d->steps;
  hlb_status st = HLB_OK;
  for (int k = 0; k < GRAPH_STEPS && st == HLB_OK; ++k) st = launch_step(d);
  const cudaError_t e = cudaStreamEndCapture(d->stream, &g);
  d->steps = s0;
  d->parity = 0;
  if (st != HLB_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return HLB_ECUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&d->graph, g, 0);
  cudaGraphDestroy(g);
  return ei == cudaSuccess ? HLB_OK : HLB_ECUDA;
}

}  // namespace

namespace {
// Whether variant v can run domain d: the row-marching kernels need nx <=
// MARCH_MAX_NX; the split step and the row-marching kernels take the
// finite-volume scheme only; the fused tiled kernel is the isotropic scheme's.
bool variant_ok(const hlb_domain* d, int v) {
  if (is_march(v)) return d->p.nx <= MARCH_MAX_NX && d->p.diffusion == HLB_DIFF_FV;
  if (is_split(v)) return d->p.diffusion == HLB_DIFF_FV;
  return true;
}

// Initial state into buffer set `par` (the other T buffer gets the same T, so
// that hlb_read after an odd number of steps finds T^n).
hlb_status set_fields_at(hlb_domain* d, const float* d_rho, const float* d_T, int par) {
  if (!d || !d_rho || !d_T) return HLB_EINVAL;
  StepArgs a = args_for(d, par);
  k_init<<<INIT_BLOCKS, 256, 0, d->stream>>>(a, d_rho, d_T, d->f[par], d->T[par], d->ftop[0], d->ftop[1]);
  k_init<<<INIT_BLOCKS, 256, 0, d->stream>>>(a, d_rho, d_T, d->f[par ^ 1], d->T[par ^ 1], nullptr, nullptr);
  k_init_state<<<1, 32, 0, d->stream>>>(d->partials, INIT_BLOCKS, d->state, 1.0 / (double)d->n_fluid);
  if (cudaGetLastError() != cudaSuccess) return HLB_ECUDA;
  d->parity = par;
  d->steps = 0;
  d->fields_set = true;
  d->host_flags = 0;
  return HLB_OK;
}

hlb_status init_domain(hlb_domain* d, const hlb_params* p, char* ws, cudaStream_t stream) {
  const Layout L = layout_of(p);
  d->p = *p;
  const PRHost e = pr_of(p);
  d->Tc = e.Tc;
  if (!(d->p.rho_l > 0 && d->p.rho_v > 0)) {
    double rl, rv;
    if (!coexistence(e, p->Ts_over_Tc * e.Tc, &rl, &rv, nullptr)) return HLB_EINVAL;
    d->p.rho_l = rl;
    d->p.rho_v = rv;
  }
  hlb_params& q = d->p;
  q.n_sub = resolved_nsub(p);
  if (!(q.rho_w > 0)) q.rho_w = 3.0 * q.rho_l;
  if (!(q.cv_w > 0)) q.cv_w = q.cv;
  if (!(q.lambda_w > 0)) q.lambda_w = 3.0 * q.rho_l * q.cv * q.k;
  d->rho_ref = q.storage == HLB_STORE_DEVIATION ? q.rho_v : 0.0;
  d->stream = stream;

  const size_t N = (size_t)q.nx * q.ny;
  d->f[0] = (float*)(ws + L.f);
  d->f[1] = d->f[0] + 9 * plane_stride(N);
  d->T[0] = (float*)(ws + L.T);
  d->T[1] = d->T[0] + N;
  d->Gw = (float*)(ws + L.Gw);
  d->ftop[0] = (float*)(ws + L.ftop);
  d->ftop[1] = d->ftop[0] + 3 * q.nx;
  d->partials = (double*)(ws + L.partials);
  d->state = (DevState*)(ws + L.state);
  d->hist = (double*)(ws + L.hist);
  d->mom = (float*)(ws + L.mom);
  d->Tscr = d->mom + 3 * N;
  d->fpart = (double*)(ws + L.fpart);
  d->epart = (double*)(ws + L.epart);
  if (q.n_sub > 1) {
    d->subpart = (double*)(ws + L.sub);
    d->sub_grid = sub_grid_of(q.nx, q.ny);
  }
  const int fluid_rows = q.ny - q.wall_rows - (q.top_bc == HLB_TOP_WALL ? 1 : 0);
  d->n_fluid = (long long)fluid_rows * q.nx;
  // the split step for the finite-volume scheme; the fused tiled kernel for the isotropic one
  set_variant_grids(d, q.diffusion == HLB_DIFF_FV ? 0 : FIRST_TILED);
  d->smem = smem_bytes();

  StepArgs& a = d->base;
  memset(&a, 0, sizeof(a));
  a.nx = q.nx;
  a.ny = q.ny;
  a.W = q.wall_rows;
  a.top_bc = q.top_bc;
  a.eos_T_fixed = q.eos_T_fixed;
  a.plane = (long long)plane_stride(N);
  a.R = (float)q.R;
  a.a = (float)q.a;
  a.b = (float)q.b;
  a.kappa = (float)e.kappa;
  a.invTc = (float)(1.0 / e.Tc);
  a.Ts = (float)(q.Ts_over_Tc * e.Tc);
  a.G = (float)q.G;
  a.g_y = (float)q.g_y;
  const double tau_e = 1.0 / q.s_e, tau_z = 1.0 / q.s_zeta;
  a.sig_e = (float)((1.0 - 0.5 * q.s_e) * q.sigma_coef * q.sigma / (tau_e - 0.5));
  a.sig_z = (float)((1.0 - 0.5 * q.s_zeta) * q.sigma_coef * q.sigma / (tau_z - 0.5));
  a.s_e = (float)q.s_e;
  a.s_z = (float)q.s_zeta;
  a.s_j = (float)q.s_j;
  a.s_q = (float)q.s_q;
  a.tau_l = (float)q.tau_l;
  a.tau_v = (float)q.tau_v;
  a.rho_v = (float)q.rho_v;
  a.dtau_drho = (float)((q.tau_l - q.tau_v) / (q.rho_l - q.rho_v));
  a.rho_ref = (float)d->rho_ref;
  a.rho_mid = (float)(0.5 * (q.rho_l + q.rho_v));
  a.cvk = (float)(q.cv * q.k);
  a.cv = (float)q.cv;
  a.rcv_w = (float)(q.rho_w * q.cv_w);
  a.inv_rcv_w = (float)(1.0 / (q.rho_w * q.cv_w));
  a.lambda_w = (float)q.lambda_w;
  a.lambda_top = (float)(q.lambda_top > 0 ? q.lambda_top : q.lambda_w);
  a.bottom_flux = q.bottom_bc == HLB_BOTTOM_FLUX ? 1 : 0;
  a.q_in = (float)q.q_in;
  a.dt = (float)(1.0 / q.n_sub);
  a.iso = q.diffusion == HLB_DIFF_ISO ? 1 : 0;
  a.kd = (float)q.k;
  a.kd_w = (float)(q.lambda_w / (q.rho_w * q.cv_w));
  a.inv_k = (float)(1.0 / q.k);
  a.T_bottom = (float)q.T_bottom;
  a.T_top = (float)q.T_top;
  a.Gw = d->Gw;
  a.partials = d->partials;
  a.state = d->state;
  a.mom = d->mom;
  a.T_scr = d->Tscr;
  a.fpart = d->fpart;
  a.epart = d->epart;

  for (int v = 0; v < NSPLIT; ++v) {
    if (cudaFuncSetAttribute(FLOWS[v].single_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FLOWS[v].smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(FLOWS[v].batch_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FLOWS[v].smem) !=
            cudaSuccess)
      return HLB_ECUDA;
  }
  for (int v = 0; v < NSPLIT; ++v) {
    if (cudaFuncSetAttribute(FLOWS[v].esingle_fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)FLOWS[v].esmem) != cudaSuccess ||
        cudaFuncSetAttribute(FLOWS[v].ebatch_fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)FLOWS[v].esmem) != cudaSuccess)
      return HLB_ECUDA;
  }
  for (int v = 0; v < NVARIANTS; ++v) {
    if (cudaFuncSetAttribute(VARIANTS[v].single_fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)VARIANTS[v].smem) != cudaSuccess ||
        cudaFuncSetAttribute(VARIANTS[v].batch_fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)VARIANTS[v].smem) != cudaSuccess)
      return HLB_ECUDA;
  }
  if (q.n_sub > 1 && cudaFuncSetAttribute(k_energy_substep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sub_smem_bytes()) != cudaSuccess)
    return HLB_ECUDA;
  if (cudaFuncSetAttribute(k_march, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)march_smem(MARCH_MAX_NX)) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_march_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)march_smem(MARCH_MAX_NX)) != cudaSuccess)
    return HLB_ECUDA;
  // uniform wetting table
  return hlb_set_nucleation_sites(d, 0, nullptr);
}

}  // namespace


// ------------------------------------------------------------------- batch
struct hlb_batch {
  int n = 0;
  std::vector<hlb_domain> dom;
  cudaStream_t stream = nullptr;
  DomArgs* d_desc = nullptr;   // [2][n]: per-domain descriptors for batch parity 0 and 1
  StepArgs phys;               // model parameters shared by the batch
  ReduceArgs* d_ra = nullptr;  // [n]
  SplitReduceArgs* d_sra = nullptr;  // [n]: the split step's reduction
  int2* d_blk = nullptr;       // [blocks]: (domain, tile within the domain) of each step block
  int2* d_eblk = nullptr;      // [energy blocks] of the split step
  std::vector<int2> eblk;      // host copy of d_eblk
  int total_etiles = 0;
  int* d_active = nullptr;     // [n]
  float2* d_lag = nullptr;     // [n]: lagged U/(1+U) and mean density, written by the reduction
  std::vector<int> tile_off;
  std::vector<int> active;
  int total_tiles = 0;
  int parity = 0;
  long long steps = 0;
  size_t smem = 0;
  int variant = 0;
  cudaGraphExec_t graph = nullptr;
  std::vector<int2> blk;  // host copy of d_blk
  // row-marching variants: one launch per group of domains with the same row
  // stride (block size), each on its own stream forked from and joined to the
  // batch stream, so that the groups' blocks share the GPU
  struct Group {
    int ns, off, count;
  };
  std::vector<Group> groups;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr;
  // split step in two lanes: domains [0, lane_split) on the batch stream,
  // [lane_split, n) on side[0], whose flow kernel of a step waits for the first
  // lane's, so that one lane's energy kernels run beside the other lane's flow
  // kernel (the flow kernel is bound by DRAM, the energy kernel by issue)
  int lanes = 1;
  int lane_split = 0, lane_blk = 0, lane_eblk = 0;  // first domain, flow block, energy block of lane B
  cudaEvent_t ev_lane = nullptr;       // lane A's flow kernel of the current step done
  cudaEvent_t ev_lane_join = nullptr;  // lane B's last work done
  bool lane_pending = false;           // lane B has work not yet joined into the batch stream
  ~hlb_batch() {
    for (cudaStream_t s : side) cudaStreamDestroy(s);
    for (cudaEvent_t e : ev_join) cudaEventDestroy(e);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_lane) cudaEventDestroy(ev_lane);
    if (ev_lane_join) cudaEventDestroy(ev_lane_join);
  }
};

namespace {

struct BatchLayout {
  std::vector<size_t> dom_off;
  size_t desc, ra, sra, blk, eblk, active, lag, total;
};

BatchLayout batch_layout(int n, const hlb_params* p) {
  BatchLayout L;
  size_t o = 0, max_blocks = 0, max_eblocks = 0;
  for (int i = 0; i < n; ++i) {
    L.dom_off.push_back(o);
    o += layout_of(p + i).total;
    const size_t tiled = (size_t)((p[i].nx + TILE_X - 1) / TILE_X) * ((p[i].ny + MIN_TILE_Y - 1) / MIN_TILE_Y);
    const size_t flow = flow_part_slots(p[i].nx, p[i].ny, p[i].wall_rows, p[i].top_bc);
    max_blocks += tiled > flow ? tiled : flow;
    const dim3 eg = energy_grid_of(p[i].nx, p[i].ny);
    max_eblocks += (size_t)eg.x * eg.y;
  }
  L.desc = o;     o += align_up(2 * (size_t)n * sizeof(DomArgs));
  L.ra = o;       o += align_up((size_t)n * sizeof(ReduceArgs));
  L.sra = o;      o += align_up((size_t)n * sizeof(SplitReduceArgs));
  L.blk = o;      o += align_up(max_blocks * sizeof(int2));
  L.eblk = o;     o += align_up(max_eblocks * sizeof(int2));
  L.active = o;   o += align_up((size_t)n * sizeof(int));
  L.lag = o;      o += align_up((size_t)n * sizeof(float2));
  L.total = o;
  return L;
}

DomArgs dom_args(const StepArgs& a) {
  DomArgs d;
  d.nx = a.nx;
  d.ny = a.ny;
  d.W = a.W;
  d.top_bc = a.top_bc;
  d.eos_T_fixed = a.eos_T_fixed;
  d.plane = a.plane;
  d.T_bottom = a.T_bottom;
  d.T_top = a.T_top;
  d.f_in = a.f_in;
  d.f_out = a.f_out;
  d.T_in = a.T_in;
  d.T_out = a.T_out;
  d.Gw = a.Gw;
  d.ftop_in = a.ftop_in;
  d.ftop_out = a.ftop_out;
  d.partials = a.partials;
  d.state = a.state;
  d.mom = a.mom;
  d.T_scr = a.T_scr;
  d.fpart = a.fpart;
  d.epart = a.epart;
  return d;
}

// The model parameters of a StepArgs (everything DomArgs does not carry).
StepArgs physics_of(const StepArgs& a) {
  StepArgs p = a;
  p.nx = p.ny = p.W = p.top_bc = p.eos_T_fixed = 0;
  p.plane = 0;
  p.T_bottom = p.T_top = 0.f;
  p.f_in = p.T_in = p.Gw = p.ftop_in = nullptr;
  p.f_out = p.T_out = p.ftop_out = nullptr;
  p.partials = nullptr;
  p.state = nullptr;
  p.mom = p.T_scr = nullptr;
  p.fpart = p.epart = nullptr;
  return p;
}

hlb_status upload_tables(hlb_batch* b) {
  std::vector<DomArgs> desc(2 * (size_t)b->n);
  std::vector<ReduceArgs> ra(b->n);
  std::vector<SplitReduceArgs> sra(b->n);
  const std::vector<int2>& blk = b->blk;
  for (int i = 0; i < b->n; ++i) {
    hlb_domain* d = &b->dom[i];
    desc[i] = dom_args(args_for(d, 0));
    desc[b->n + i] = dom_args(args_for(d, 1));
    ra[i].partials = d->partials;
    ra[i].state = d->state;
    ra[i].hist = d->hist;
    ra[i].nblk = (int)(d->grid.x * d->grid.y);
    ra[i].inv_nfluid = 1.0 / (double)d->n_fluid;
    ra[i].inv_nx = 1.0 / (double)d->p.nx;
    sra[i].fpart = d->fpart;
    sra[i].epart = d->epart;
    sra[i].state = d->state;
    sra[i].hist = d->hist;
    sra[i].nf = (int)(d->grid.x * d->grid.y);
    sra[i].ne = (int)(d->egrid.x * d->egrid.y);
    sra[i].inv_nfluid = ra[i].inv_nfluid;
    sra[i].inv_nx = ra[i].inv_nx;
  }
  if (cudaMemcpyAsync(b->d_desc, desc.data(), desc.size() * sizeof(DomArgs), cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(b->d_ra, ra.data(), ra.size() * sizeof(ReduceArgs), cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(b->d_sra, sra.data(), sra.size() * sizeof(SplitReduceArgs), cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess ||
      cudaMemcpyAsync(b->d_blk, blk.data(), blk.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess ||
      (!b->eblk.empty() && cudaMemcpyAsync(b->d_eblk, b->eblk.data(), b->eblk.size() * sizeof(int2),
                                           cudaMemcpyHostToDevice, b->stream) != cudaSuccess) ||
      cudaMemcpyAsync(b->d_active, b->active.data(), b->active.size() * sizeof(int), cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess)
    return HLB_ECUDA;
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? HLB_OK : HLB_ECUDA;
}

// One batched step.  Events (any may be null): `before` the step kernels,
// `mid` after the flow kernel of a split step, `after` the step kernels
// (before the reduction).
// Make the batch stream wait for everything lane B has been given.
hlb_status lane_join(hlb_batch* b) {
  if (!b->lane_pending) return HLB_OK;
  if (cudaEventRecord(b->ev_lane_join, b->side[0]) != cudaSuccess ||
      cudaStreamWaitEvent(b->stream, b->ev_lane_join, 0) != cudaSuccess)
    return HLB_ECUDA;
  b->lane_pending = false;
  return HLB_OK;
}

bool two_lanes(const hlb_batch* b) { return is_split(b->variant) && b->lanes == 2 && b->n >= 2; }

// One split step in two lanes (see hlb_batch::lanes); lane B is left pending.
hlb_status batch_launch_lanes(hlb_batch* b, const DomArgs* desc) {
  const FlowVariant& fv = FLOWS[b->variant];
  const int nsub = b->dom[0].p.n_sub;
  const int m = b->lane_split;
  cudaStream_t a = b->stream, s2 = b->side[0];
  fv.launch_batch(b->lane_blk, fv.smem, a, b->phys, desc, b->d_blk, b->d_active, b->d_lag);
  if (cudaEventRecord(b->ev_lane, a) != cudaSuccess) return HLB_ECUDA;
  for (int s = 1; s <= nsub; ++s) fv.energy_batch(b->lane_eblk, a, b->phys, desc, b->d_eblk, b->d_active, s, nsub);
  k_reduce_split_batch<<<m, 256, 0, a>>>(b->d_sra, b->d_active, b->d_lag, HIST_CAP);
  if (cudaStreamWaitEvent(s2, b->ev_lane, 0) != cudaSuccess) return HLB_ECUDA;
  fv.launch_batch(b->total_tiles - b->lane_blk, fv.smem, s2, b->phys, desc, b->d_blk + b->lane_blk, b->d_active,
                  b->d_lag);
  for (int s = 1; s <= nsub; ++s)
    fv.energy_batch(b->total_etiles - b->lane_eblk, s2, b->phys, desc, b->d_eblk + b->lane_eblk, b->d_active, s,
                    nsub);
  k_reduce_split_batch<<<b->n - m, 256, 0, s2>>>(b->d_sra + m, b->d_active + m, b->d_lag + m, HIST_CAP);
  b->lane_pending = true;
  return cudaGetLastError() == cudaSuccess ? HLB_OK : HLB_ECUDA;
}

hlb_status batch_launch(hlb_batch* b, cudaEvent_t before, cudaEvent_t after, cudaEvent_t mid = nullptr) {
  if (before && cudaEventRecord(before, b->stream) != cudaSuccess) return HLB_ECUDA;
  const DomArgs* desc = b->d_desc + (size_t)b->parity * b->n;
  if (two_lanes(b)) {
    // the flow/energy boundary is not a point in time here: `mid` is not recorded
    hlb_status st = batch_launch_lanes(b, desc);
    if (st == HLB_OK && after) st = lane_join(b);
    if (st != HLB_OK) return st;
    if (after && cudaEventRecord(after, b->stream) != cudaSuccess) return HLB_ECUDA;
    b->parity ^= 1;
    b->steps += 1;
    for (int i = 0; i < b->n; ++i) {
      if (b->active[i]) {
        b->dom[i].parity ^= 1;
        b->dom[i].steps += 1;
      }
    }
    return HLB_OK;
  }
  if (is_split(b->variant)) {
    const FlowVariant& fv = FLOWS[b->variant];
    fv.launch_batch(b->total_tiles, fv.smem, b->stream, b->phys, desc, b->d_blk, b->d_active, b->d_lag);
    if (mid && cudaEventRecord(mid, b->stream) != cudaSuccess) return HLB_ECUDA;
    const int nsub = b->dom[0].p.n_sub;
    for (int s = 1; s <= nsub; ++s)
      fv.energy_batch(b->total_etiles, b->stream, b->phys, desc, b->d_eblk, b->d_active, s, nsub);
    if (after && cudaEventRecord(after, b->stream) != cudaSuccess) return HLB_ECUDA;
    k_reduce_split_batch<<<b->n, 256, 0, b->stream>>>(b->d_sra, b->d_active, b->d_lag, HIST_CAP);
    if (cudaGetLastError() != cudaSuccess) return HLB_ECUDA;
    b->parity ^= 1;
    b->steps += 1;
    for (int i = 0; i < b->n; ++i) {
      if (b->active[i]) {
        b->dom[i].parity ^= 1;
        b->dom[i].steps += 1;
      }
    }
    return HLB_OK;
  }
  if (is_march(b->variant)) {
    const int S = march_seg(b->variant);
    if (cudaEventRecord(b->ev_fork, b->stream) != cudaSuccess) return HLB_ECUDA;
    for (size_t g = 0; g < b->groups.size(); ++g) {
      const hlb_batch::Group& G = b->groups[g];
      if (cudaStreamWaitEvent(b->side[g], b->ev_fork, 0) != cudaSuccess) return HLB_ECUDA;
      k_march_batch<<<G.count, G.ns, march_smem(G.ns), b->side[g]>>>(b->phys, desc, b->d_blk + G.off, b->d_active,
                                                                    b->d_lag, S);
      if (cudaEventRecord(b->ev_join[g], b->side[g]) != cudaSuccess ||
          cudaStreamWaitEvent(b->stream, b->ev_join[g], 0) != cudaSuccess)
        return HLB_ECUDA;
    }
  } else {
    const Variant& tv = VARIANTS[tiled_index(b->variant)];
    tv.launch_batch(b->total_tiles, tv.smem, b->stream, b->phys, desc, b->d_blk, b->d_active, b->d_lag);
  }
  if (after && cudaEventRecord(after, b->stream) != cudaSuccess) return HLB_ECUDA;
  k_reduce_batch<<<b->n, 256, 0, b->stream>>>(b->d_ra, b->d_active, b->d_lag, HIST_CAP);
  if (cudaGetLastError() != cudaSuccess) return HLB_ECUDA;
  b->parity ^= 1;
  b->steps += 1;
  for (int i = 0; i < b->n; ++i) {
    if (b->active[i]) {
      b->dom[i].parity ^= 1;
      b->dom[i].steps += 1;
    }
  }
  return HLB_OK;
}

void batch_drop_graph(hlb_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

hlb_status batch_build_graph(hlb_batch* b) {
  if (b->parity != 0) return HLB_ESTATE;
  std::vector<int> par(b->n);
  std::vector<long long> stp(b->n);
  for (int i = 0; i < b->n; ++i) {
    par[i] = b->dom[i].parity;
    stp[i] = b->dom[i].steps;
  }
  const long long s0 = b->steps;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HLB_ECUDA;
  hlb_status st = HLB_OK;
  for (int k = 0; k < GRAPH_STEPS && st == HLB_OK; ++k) st = batch_launch(b, nullptr, nullptr);
  if (st == HLB_OK) st = lane_join(b);  // a capture ends with every forked stream joined
  const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  b->steps = s0;
  b->parity = 0;
  for (int i = 0; i < b->n; ++i) {
    b->dom[i].parity = par[i];
    b->dom[i].steps = stp[i];
  }
  if (st != HLB_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return HLB_ECUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  return ei == cudaSuccess ? HLB_OK : HLB_ECUDA;
}

bool batch_ok(const hlb_batch* b, int i) { return b && i >= 0 && i < b->n; }

bool batch_march_ok(const hlb_batch* b) {
  for (int i = 0; i < b->n; ++i)
    if (b->dom[i].p.nx > MARCH_MAX_NX) return false;
  return true;
}

// Select variant v for every domain of the batch: block table (grouped by row
// stride for the row-marching variants), side streams, device tables.
bool batch_variant_ok(const hlb_batch* b, int v) {
  if (is_march(v) && !batch_march_ok(b)) return false;
  // energy sub-steps (Eq. 27) run only in the split form
  if (!is_split(v) && b->dom[0].p.n_sub > 1) return false;
  return true;
}

// Lane B of the two-lane split step: the domains from the first one at which
// the cells of lane A reach half of the batch's, their flow and energy blocks;
// a side stream and the two events.
hlb_status lane_setup(hlb_batch* b) {
  if (!is_split(b->variant) || b->n < 2) return HLB_OK;
  double total = 0.0, acc = 0.0;
  for (int i = 0; i < b->n; ++i) total += (double)b->dom[i].p.nx * b->dom[i].p.ny;
  int m = 1;
  for (int i = 0; i < b->n - 1; ++i) {
    acc += (double)b->dom[i].p.nx * b->dom[i].p.ny;
    m = i + 1;
    if (acc >= 0.5 * total) break;
  }
  b->lane_split = m;
  b->lane_blk = b->tile_off[m];
  int e = 0;
  while (e < (int)b->eblk.size() && b->eblk[e].x < m) ++e;
  b->lane_eblk = e;
  if (b->side.empty()) {
    cudaStream_t s2 = nullptr;
    cudaEvent_t ej = nullptr;
    if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess) return HLB_ECUDA;
    b->side.push_back(s2);
    if (cudaEventCreateWithFlags(&ej, cudaEventDisableTiming) != cudaSuccess) return HLB_ECUDA;
    b->ev_join.push_back(ej);
  }
  if (!b->ev_lane && cudaEventCreateWithFlags(&b->ev_lane, cudaEventDisableTiming) != cudaSuccess) return HLB_ECUDA;
  if (!b->ev_lane_join && cudaEventCreateWithFlags(&b->ev_lane_join, cudaEventDisableTiming) != cudaSuccess)
    return HLB_ECUDA;
  return HLB_OK;
}

hlb_status set_batch_variant(hlb_batch* b, int v) {
  if (!batch_variant_ok(b, v)) return HLB_EINVAL;
  const hlb_status sj = lane_join(b);
  if (sj != HLB_OK) return sj;
  b->variant = v;
  b->tile_off.assign(b->n + 1, 0);
  for (int i = 0; i < b->n; ++i) {
    hlb_domain* d = &b->dom[i];
    set_variant_grids(d, v);
    b->tile_off[i + 1] = b->tile_off[i] + (int)(d->grid.x * d->grid.y);
  }
  b->total_tiles = b->tile_off[b->n];
  b->blk.clear();
  b->eblk.clear();
  b->groups.clear();
  if (is_split(v)) {
    for (int i = 0; i < b->n; ++i) {
      const dim3 eg = b->dom[i].egrid;
      for (int t = 0; t < (int)(eg.x * eg.y); ++t) b->eblk.push_back(make_int2(i, t));
    }
  }
  b->total_etiles = (int)b->eblk.size();
  if (is_march(v)) {
    std::vector<int> strides;
    for (int i = 0; i < b->n; ++i) {
      const int ns = march_row_stride(b->dom[i].p.nx);
      bool seen = false;
      for (int s2 : strides) seen = seen || s2 == ns;
      if (!seen) strides.push_back(ns);
    }
    // widest first: their blocks are the largest and the longest
    for (size_t a = 0; a < strides.size(); ++a)
      for (size_t c = a + 1; c < strides.size(); ++c)
        if (strides[c] > strides[a]) std::swap(strides[a], strides[c]);
    for (int ns : strides) {
      hlb_batch::Group G{ns, (int)b->blk.size(), 0};
      for (int i = 0; i < b->n; ++i) {
        if (march_row_stride(b->dom[i].p.nx) != ns) continue;
        for (int t = 0; t < (int)b->dom[i].grid.x; ++t) b->blk.push_back(make_int2(i, t));
      }
      G.count = (int)b->blk.size() - G.off;
      b->groups.push_back(G);
    }
    if (!b->ev_fork && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess)
      return HLB_ECUDA;
    while (b->side.size() < b->groups.size()) {
      cudaStream_t s2 = nullptr;
      cudaEvent_t e = nullptr;
      if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess) return HLB_ECUDA;
      b->side.push_back(s2);
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return HLB_ECUDA;
      b->ev_join.push_back(e);
    }
  } else {
    for (int i = 0; i < b->n; ++i)
      for (int t = b->tile_off[i]; t < b->tile_off[i + 1]; ++t) b->blk.push_back(make_int2(i, t - b->tile_off[i]));
  }
  b->smem = is_split(v) ? FLOWS[v].smem : (is_march(v) ? march_smem(MARCH_MAX_NX) : VARIANTS[tiled_index(v)].smem);
  const hlb_status st = lane_setup(b);
  if (st != HLB_OK) return st;
  batch_drop_graph(b);
  return upload_tables(b);
}

// ------------------------------------------------------------ checkpoints
// Byte image of a domain's carried state (layout in include/hlb.h).
constexpr unsigned long long CKPT_MAGIC = 0x3154504b43424c48ull;  // "HLBCKPT1" read little-endian
constexpr int CKPT_VERSION = 1;
constexpr size_t CKPT_HEADER = 512;

struct CkptHeader {
  unsigned long long magic;
  int version, header_bytes, state_bytes;
  int nx, ny, wall_rows, top_bc, bottom_bc, storage, hist_len;
  double rho_ref, T_bottom;
  long long step;
  DevState state;
};
static_assert(sizeof(CkptHeader) <= CKPT_HEADER, "checkpoint header does not fit its slot");

// float offsets of the arrays after the header
struct CkptLayout {
  size_t f, T, T_prev, ftop, Gw, hist;  // hist is a byte offset, 8-byte aligned
};

CkptLayout ckpt_layout(int nx, int ny) {
  const size_t N = (size_t)nx * ny;
  CkptLayout L;
  L.f = 0;
  L.T = L.f + 9 * N;
  L.T_prev = L.T + N;
  L.ftop = L.T_prev + N;
  L.Gw = L.ftop + 3 * (size_t)nx;
  L.hist = (CKPT_HEADER + (L.Gw + nx) * sizeof(float) + 7) & ~(size_t)7;
  return L;
}

hlb_status ckpt_save(hlb_domain* d, void* h_buf, size_t cap, size_t* h_len) {
  if (!d || !h_buf || !h_len) return HLB_EINVAL;
  if (!d->fields_set) return HLB_ESTATE;
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  if (cudaMemcpyAsync(&h.state, d->state, sizeof(DevState), cudaMemcpyDeviceToHost, d->stream) != cudaSuccess ||
      cudaStreamSynchronize(d->stream) != cudaSuccess)
    return HLB_ECUDA;
  const int nx = d->p.nx, ny = d->p.ny;
  const CkptLayout L = ckpt_layout(nx, ny);
  const int hist_len = h.state.hist_len < 0 ? 0 : (h.state.hist_len > HIST_CAP ? HIST_CAP : h.state.hist_len);
  const size_t need = L.hist + (size_t)hist_len * sizeof(double);
  if (cap < need) return HLB_EINVAL;
  h.magic = CKPT_MAGIC;
  h.version = CKPT_VERSION;
  h.header_bytes = (int)CKPT_HEADER;
  h.state_bytes = (int)sizeof(DevState);
  h.nx = nx;
  h.ny = ny;
  h.wall_rows = d->p.wall_rows;
  h.top_bc = d->p.top_bc;
  h.bottom_bc = d->p.bottom_bc;
  h.storage = d->p.storage;
  h.hist_len = hist_len;
  h.rho_ref = d->rho_ref;
  h.T_bottom = d->p.T_bottom;
  h.step = h.state.step;
  char* out = (char*)h_buf;
  memset(out, 0, CKPT_HEADER);
  memcpy(out, &h, sizeof(h));
  float* a = (float*)(out + CKPT_HEADER);
  const size_t N = (size_t)nx * ny;
  const int cur = d->parity;
  cudaStream_t s = d->stream;
  if (cudaMemcpy2DAsync(a + L.f, N * sizeof(float), d->f[cur], (size_t)d->base.plane * sizeof(float),
                        N * sizeof(float), 9, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(a + L.T, d->T[cur], N * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(a + L.T_prev, d->T[cur ^ 1], N * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(a + L.ftop, d->ftop[cur], 3 * (size_t)nx * sizeof(float), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(a + L.Gw, d->Gw, (size_t)nx * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      (hist_len > 0 && cudaMemcpyAsync(out + L.hist, d->hist, (size_t)hist_len * sizeof(double),
                                       cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return HLB_ECUDA;
  *h_len = need;
  return HLB_OK;
}

// Restore into buffer set `par` (the populations and the outlet memory go to
// both sets, so that every buffer a later step may read holds saved values).
hlb_status ckpt_load(hlb_domain* d, const void* h_buf, size_t len, int par) {
  if (!d || !h_buf || len < CKPT_HEADER) return HLB_EINVAL;
  CkptHeader h;
  memcpy(&h, h_buf, sizeof(h));
  const hlb_params& p = d->p;
  if (h.magic != CKPT_MAGIC || h.version != CKPT_VERSION || h.header_bytes != (int)CKPT_HEADER ||
      h.state_bytes != (int)sizeof(DevState))
    return HLB_EINVAL;
  if (h.nx != p.nx || h.ny != p.ny || h.wall_rows != p.wall_rows || h.top_bc != p.top_bc ||
      h.bottom_bc != p.bottom_bc || h.storage != p.storage || memcmp(&h.rho_ref, &d->rho_ref, sizeof(double)) != 0)
    return HLB_EINVAL;
  if (h.hist_len < 0 || h.hist_len > HIST_CAP || h.state.hist_len != h.hist_len || h.step < 0 ||
      h.state.step != h.step || !isfinite(h.T_bottom))
    return HLB_EINVAL;
  const CkptLayout L = ckpt_layout(p.nx, p.ny);
  if (len < L.hist + (size_t)h.hist_len * sizeof(double)) return HLB_EINVAL;
  const char* in = (const char*)h_buf;
  const float* a = (const float*)(in + CKPT_HEADER);
  const size_t N = (size_t)p.nx * p.ny;
  cudaStream_t s = d->stream;
  bool ok = cudaStreamSynchronize(s) == cudaSuccess;
  for (int k = 0; k < 2 && ok; ++k) {
    ok = cudaMemcpy2DAsync(d->f[k], (size_t)d->base.plane * sizeof(float), a + L.f, N * sizeof(float),
                           N * sizeof(float), 9, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(d->ftop[k], a + L.ftop, 3 * (size_t)p.nx * sizeof(float), cudaMemcpyHostToDevice, s) ==
             cudaSuccess;
  }
  ok = ok &&
       cudaMemcpyAsync(d->T[par], a + L.T, N * sizeof(float), cudaMemcpyHostToDevice, s) == cudaSuccess &&
       cudaMemcpyAsync(d->T[par ^ 1], a + L.T_prev, N * sizeof(float), cudaMemcpyHostToDevice, s) == cudaSuccess &&
       cudaMemcpyAsync(d->Gw, a + L.Gw, (size_t)p.nx * sizeof(float), cudaMemcpyHostToDevice, s) == cudaSuccess &&
       (h.hist_len == 0 || cudaMemcpyAsync(d->hist, in + L.hist, (size_t)h.hist_len * sizeof(double),
                                           cudaMemcpyHostToDevice, s) == cudaSuccess) &&
       cudaMemcpyAsync(d->state, &h.state, sizeof(DevState), cudaMemcpyHostToDevice, s) == cudaSuccess &&
       cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) return HLB_ECUDA;
  d->parity = par;
  d->steps = h.step;
  d->fields_set = true;
  d->host_flags = h.state.error_flags;
  return hlb_set_wall(d, h.T_bottom);
}

}  // namespace

extern "C" {

void hlb_params_default(hlb_params* p, int nx, int ny) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->nx = nx;
  p->ny = ny;
  p->wall_rows = 1;
  p->top_bc = HLB_TOP_WALL;
  p->eos_T_fixed = 0;
  p->n_sub = 1;
  p->storage = HLB_STORE_DEVIATION;
  p->a = 3.0 / 49.0;
  p->b = 2.0 / 21.0;
  p->R = 1.0;
  p->omega = 0.344;
  p->Ts_over_Tc = 0.86;
  p->G = -1.0;
  p->sigma = 0.107;
  p->sigma_coef = 12.0;
  p->s_rho = 1.0;
  p->s_e = 0.8;
  p->s_zeta = 0.8;
  p->s_j = 1.0;
  p->s_q = 1.1;
  p->tau_l = 0.8;
  p->tau_v = 1.0;
  p->cv = 6.0;
  p->k = 0.1;
  p->rho_w = 0.0;
  p->cv_w = 0.0;
  p->lambda_w = 0.0;
  p->g_y = 0.0;
  p->Gw0 = 0.3;
  p->T_bottom = 0.0;
  p->T_top = 0.0;
  p->rho_l = 0.0;
  p->rho_v = 0.0;
}

hlb_status hlb_eos_coexistence(const hlb_params* p, double* Tc, double* rho_l, double* rho_v, double* h_fg) {
  if (!p || !(p->a > 0 && p->b > 0 && p->R > 0 && p->Ts_over_Tc > 0)) return HLB_EINVAL;
  const PRHost e = pr_of(p);
  if (Tc) *Tc = e.Tc;
  double rl, rv, h;
  if (!coexistence(e, p->Ts_over_Tc * e.Tc, &rl, &rv, &h)) return HLB_EINVAL;
  if (rho_l) *rho_l = rl;
  if (rho_v) *rho_v = rv;
  if (h_fg) *h_fg = h;
  return HLB_OK;
}

size_t hlb_workspace_bytes(const hlb_params* p) {
  if (!params_valid(p)) return 0;
  return layout_of(p).total;
}

hlb_status hlb_init(hlb_domain** out, const hlb_params* p, void* d_workspace, size_t workspace_bytes, void* stream) {
  if (!out || !params_valid(p) || !d_workspace) return HLB_EINVAL;
  *out = nullptr;
  if (((uintptr_t)d_workspace & 255) != 0) return HLB_EINVAL;
  if (workspace_bytes < layout_of(p).total) return HLB_EINVAL;
  hlb_domain* d = new (std::nothrow) hlb_domain();
  if (!d) return HLB_EINVAL;
  const hlb_status st = init_domain(d, p, (char*)d_workspace, (cudaStream_t)stream);
  if (st != HLB_OK) {
    delete d;
    return st;
  }
  *out = d;
  return HLB_OK;
}

hlb_status hlb_set_fields(hlb_domain* d, const float* d_rho, const float* d_T) {
  return set_fields_at(d, d_rho, d_T, 0);
}

hlb_status hlb_set_wall(hlb_domain* d, double T_bottom) {
  if (!d || !isfinite(T_bottom)) return HLB_EINVAL;
  d->p.T_bottom = T_bottom;
  d->base.T_bottom = (float)T_bottom;
  drop_graph(d);
  return HLB_OK;
}

hlb_status hlb_set_nucleation_sites(hlb_domain* d, int n, const hlb_site* sites) {
  if (!d || n < 0 || (n > 0 && !sites)) return HLB_EINVAL;
  const int nx = d->p.nx;
  float* tab = (float*)malloc(sizeof(float) * nx);
  if (!tab) return HLB_EINVAL;
  for (int x = 0; x < nx; ++x) {
    double g = d->p.Gw0;
    for (int s = 0; s < n; ++s) {
      const double half = 0.5 * sites[s].width;
      if (!(half > 0)) {
        free(tab);
        return HLB_EINVAL;
      }
      double dist = fabs((double)x - sites[s].x_center);
      dist = fmin(dist, (double)nx - dist);
      if (dist <= half) {
        const double v = sites[s].gw_min + (d->p.Gw0 - sites[s].gw_min) * dist / half;
        g = fmin(g, v);
      }
    }
    tab[x] = (float)g;
  }
  const cudaError_t e = cudaMemcpyAsync(d->Gw, tab, sizeof(float) * nx, cudaMemcpyHostToDevice, d->stream);
  const cudaError_t e2 = cudaStreamSynchronize(d->stream);
  free(tab);
  return (e == cudaSuccess && e2 == cudaSuccess) ? HLB_OK : HLB_ECUDA;
}

hlb_status hlb_step(hlb_domain* d, int nsteps) {
  if (!d || nsteps < 0) return HLB_EINVAL;
  if (!d->fields_set) return HLB_ESTATE;
  if (d->host_flags) return HLB_ESTATE;
  hlb_status st = HLB_OK;
  const bool graphs = d->stream != nullptr;
  while (nsteps > 0 && st == HLB_OK) {
    if (graphs && d->parity == 0 && nsteps >= GRAPH_STEPS) {
      if (!d->graph) {
        st = build_graph(d);
        if (st != HLB_OK) return st;
      }
      if (cudaGraphLaunch(d->graph, d->stream) != cudaSuccess) return HLB_ECUDA;
      d->steps += GRAPH_STEPS;
      nsteps -= GRAPH_STEPS;
    } else {
      st = launch_step(d);
      nsteps -= 1;
    }
  }
  return st;
}

hlb_status hlb_read(hlb_domain* d, float* d_rho, float* d_ux, float* d_uy, float* d_T) {
  if (!d) return HLB_EINVAL;
  if (!d->fields_set) return HLB_ESTATE;
  const int cur = d->parity;
  StepArgs a = args_for(d, cur ^ 1);
  // args_for(cur ^ 1) has f_out = f[cur] (the current populations)
  if (d_rho || d_ux || d_uy) {
    const float* Tn = d->T[cur ^ 1];  // T^n: the temperature the last step started from
    k_read<<<INIT_BLOCKS, 256, 0, d->stream>>>(a, d->steps == 0 ? d->T[cur] : Tn, d->steps == 0 ? 1 : 0, d_rho,
                                                d_ux, d_uy);
  }
  if (d_T) {
    if (cudaMemcpyAsync(d_T, d->T[cur], sizeof(float) * (size_t)d->p.nx * d->p.ny, cudaMemcpyDeviceToDevice,
                        d->stream) != cudaSuccess)
      return HLB_ECUDA;
  }
  return cudaGetLastError() == cudaSuccess ? HLB_OK : HLB_ECUDA;
}

hlb_status hlb_diag(hlb_domain* d, hlb_diag_record* out) {
  if (!d || !out) return HLB_EINVAL;
  DevState s;
  if (cudaMemcpyAsync(&s, d->state, sizeof(s), cudaMemcpyDeviceToHost, d->stream) != cudaSuccess) return HLB_ECUDA;
  if (cudaStreamSynchronize(d->stream) != cudaSuccess) return HLB_ECUDA;
  out->step = s.step;
  out->mass = s.mass;
  out->energy = s.energy;
  out->q_bottom = s.q_bottom;
  out->q_top = s.q_top;
  out->q_interface = s.q_interface;
  out->rho_ave = s.rho_ave;
  out->u_top = s.u_top;
  out->q_bottom_timeavg = s.q_count > 0 ? s.q_sum / (double)s.q_count : 0.0;
  out->vapour_coverage = s.vcov;
  out->vapour_coverage_timeavg = s.q_count > 0 ? s.vcov_sum / (double)s.q_count : 0.0;
  out->error_flags = s.error_flags;
  d->host_flags = s.error_flags;
  if (s.error_flags & ERR_TIMEOUT) return HLB_ETIMEOUT;
  return s.error_flags ? HLB_EUNSTABLE : HLB_OK;
}

hlb_status hlb_reset_timeavg(hlb_domain* d) {
  if (!d) return HLB_EINVAL;
  const size_t off_sum = offsetof(DevState, q_sum);
  const size_t len = offsetof(DevState, error_flags) - off_sum;  // q_sum, q_count, vcov, vcov_sum
  if (cudaMemsetAsync((char*)d->state + off_sum, 0, len, d->stream) != cudaSuccess) return HLB_ECUDA;
  return HLB_OK;
}

hlb_status hlb_destroy(hlb_domain* d) {
  if (!d) return HLB_EINVAL;
  drop_graph(d);
  delete d;
  return HLB_OK;
}

int hlb_stable_substeps(const hlb_params* p) {
  if (!p || !(p->k > 0 && p->cv > 0 && p->a > 0 && p->b > 0 && p->R > 0 && p->Ts_over_Tc > 0)) return 0;
  return stable_substeps(p);
}

size_t hlb_checkpoint_bytes(const hlb_params* p) {
  if (!params_valid(p)) return 0;
  return ckpt_layout(p->nx, p->ny).hist + (size_t)HIST_CAP * sizeof(double);
}

hlb_status hlb_checkpoint_save(hlb_domain* d, void* h_buf, size_t cap, size_t* h_len) {
  return ckpt_save(d, h_buf, cap, h_len);
}

hlb_status hlb_checkpoint_load(hlb_domain* d, const void* h_buf, size_t len) {
  // a single domain resumes at buffer parity 0, where its step graph starts
  return ckpt_load(d, h_buf, len, 0);
}

// ------------------------------------------------------------- batch API
size_t hlb_batch_workspace_bytes(int n, const hlb_params* p) {
  if (n < 1 || !p) return 0;
  for (int i = 0; i < n; ++i)
    if (!params_valid(p + i) || p[i].diffusion != HLB_DIFF_FV) return 0;
  return batch_layout(n, p).total;
}

hlb_status hlb_batch_init(hlb_batch** out, int n, const hlb_params* p, void* d_workspace, size_t workspace_bytes,
                          void* stream) {
  if (!out || n < 1 || !p || !d_workspace) return HLB_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!params_valid(p + i) || p[i].diffusion != HLB_DIFF_FV) return HLB_EINVAL;
  if (((uintptr_t)d_workspace & 255) != 0) return HLB_EINVAL;
  const BatchLayout L = batch_layout(n, p);
  if (workspace_bytes < L.total) return HLB_EINVAL;
  hlb_batch* b = new (std::nothrow) hlb_batch();
  if (!b) return HLB_EINVAL;
  b->n = n;
  b->stream = (cudaStream_t)stream;
  b->dom.resize(n);
  char* ws = (char*)d_workspace;
  b->tile_off.assign(n + 1, 0);
  b->active.assign(n, 1);
  for (int i = 0; i < n; ++i) {
    const hlb_status st = init_domain(&b->dom[i], p + i, ws + L.dom_off[i], b->stream);
    if (st != HLB_OK) {
      delete b;
      return st;
    }
    b->tile_off[i + 1] = b->tile_off[i] + (int)(b->dom[i].grid.x * b->dom[i].grid.y);
  }
  b->total_tiles = b->tile_off[n];
  b->phys = physics_of(b->dom[0].base);
  for (int i = 1; i < n; ++i) {
    const StepArgs pi = physics_of(b->dom[i].base);
    if (memcmp(&pi, &b->phys, sizeof(StepArgs)) != 0) {
      delete b;  // a batch shares its model parameters; domains differ in geometry and walls
      return HLB_EINVAL;
    }
  }
  b->d_desc = (DomArgs*)(ws + L.desc);
  b->d_ra = (ReduceArgs*)(ws + L.ra);
  b->d_sra = (SplitReduceArgs*)(ws + L.sra);
  b->d_blk = (int2*)(ws + L.blk);
  b->d_eblk = (int2*)(ws + L.eblk);
  b->d_active = (int*)(ws + L.active);
  b->d_lag = (float2*)(ws + L.lag);
  const hlb_status st = set_batch_variant(b, 0);
  if (st != HLB_OK) {
    delete b;
    return st;
  }
  *out = b;
  return HLB_OK;
}

hlb_status hlb_batch_set_fields(hlb_batch* b, int i, const float* d_rho, const float* d_T) {
  if (!batch_ok(b, i)) return HLB_EINVAL;
  // the domain joins the batch at the batch's current buffer parity
  const hlb_status st = set_fields_at(&b->dom[i], d_rho, d_T, b->parity);
  if (st != HLB_OK) return st;
  k_lag_from_state<<<1, 32, 0, b->stream>>>(b->dom[i].state, b->d_lag + i);
  if (cudaGetLastError() != cudaSuccess) return HLB_ECUDA;
  if (!b->active[i]) {
    b->active[i] = 1;
    const int one = 1;
    if (cudaMemcpyAsync(b->d_active + i, &one, sizeof(int), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
      return HLB_ECUDA;
  }
  return HLB_OK;
}

hlb_status hlb_batch_set_wall(hlb_batch* b, int i, double T_bottom) {
  if (!batch_ok(b, i)) return HLB_EINVAL;
  const hlb_status st = hlb_set_wall(&b->dom[i], T_bottom);
  if (st != HLB_OK) return st;
  batch_drop_graph(b);
  return upload_tables(b);
}

hlb_status hlb_batch_set_nucleation_sites(hlb_batch* b, int i, int n, const hlb_site* h_sites) {
  if (!batch_ok(b, i)) return HLB_EINVAL;
  return hlb_set_nucleation_sites(&b->dom[i], n, h_sites);
}

hlb_status hlb_batch_step(hlb_batch* b, int nsteps) {
  if (!b || nsteps < 0) return HLB_EINVAL;
  for (int i = 0; i < b->n; ++i)
    if (!b->dom[i].fields_set) return HLB_ESTATE;
  hlb_status st = HLB_OK;
  const bool graphs = b->stream != nullptr;
  while (nsteps > 0 && st == HLB_OK) {
    if (graphs && b->parity == 0 && nsteps >= GRAPH_STEPS) {
      // the graph's lane-B kernels are not on the side stream: join it first
      st = lane_join(b);
      if (st != HLB_OK) return st;
      if (!b->graph) {
        st = batch_build_graph(b);
        if (st != HLB_OK) return st;
      }
      if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return HLB_ECUDA;
      b->steps += GRAPH_STEPS;
      for (int i = 0; i < b->n; ++i) {
        if (b->active[i]) b->dom[i].steps += GRAPH_STEPS;  // parity unchanged (even count)
      }
      nsteps -= GRAPH_STEPS;
    } else {
      st = batch_launch(b, nullptr, nullptr);
      nsteps -= 1;
    }
  }
  const hlb_status sj = lane_join(b);
  return st != HLB_OK ? st : sj;
}

hlb_status hlb_batch_set_lanes(hlb_batch* b, int lanes) {
  if (!b || (lanes != 1 && lanes != 2)) return HLB_EINVAL;
  const hlb_status st = lane_join(b);
  if (st != HLB_OK) return st;
  b->lanes = lanes;
  batch_drop_graph(b);
  return lane_setup(b);
}

hlb_status hlb_batch_step_profiled(hlb_batch* b, void* ev_before, void* ev_after) {
  if (!b) return HLB_EINVAL;
  for (int i = 0; i < b->n; ++i)
    if (!b->dom[i].fields_set) return HLB_ESTATE;
  const hlb_status st = batch_launch(b, (cudaEvent_t)ev_before, (cudaEvent_t)ev_after);
  const hlb_status sj = lane_join(b);
  return st != HLB_OK ? st : sj;
}

hlb_status hlb_batch_step_phases(hlb_batch* b, void* ev_before, void* ev_flow, void* ev_after) {
  if (!b) return HLB_EINVAL;
  for (int i = 0; i < b->n; ++i)
    if (!b->dom[i].fields_set) return HLB_ESTATE;
  const hlb_status st = batch_launch(b, (cudaEvent_t)ev_before, (cudaEvent_t)ev_after, (cudaEvent_t)ev_flow);
  const hlb_status sj = lane_join(b);
  return st != HLB_OK ? st : sj;
}

hlb_status hlb_batch_read(hlb_batch* b, int i, float* d_rho, float* d_ux, float* d_uy, float* d_T) {
  if (!batch_ok(b, i)) return HLB_EINVAL;
  return hlb_read(&b->dom[i], d_rho, d_ux, d_uy, d_T);
}

hlb_status hlb_batch_diag(hlb_batch* b, int i, hlb_diag_record* h_out) {
  if (!batch_ok(b, i)) return HLB_EINVAL;
  return hlb_diag(&b->dom[i], h_out);
}

hlb_status hlb_flux_history(hlb_domain* d, double* h_out, int max_len, int* h_len) {
  if (!d || !h_out || max_len < 0 || !h_len) return HLB_EINVAL;
  DevState s;
  if (cudaMemcpyAsync(&s, d->state, sizeof(s), cudaMemcpyDeviceToHost, d->stream) != cudaSuccess ||
      cudaStreamSynchronize(d->stream) != cudaSuccess)
    return HLB_ECUDA;
  const int len = s.hist_len < max_len ? s.hist_len : max_len;
  if (len > 0 && (cudaMemcpyAsync(h_out, d->hist, sizeof(double) * len, cudaMemcpyDeviceToHost, d->stream) !=
                      cudaSuccess ||
                  cudaStreamSynchronize(d->stream) != cudaSuccess))
    return HLB_ECUDA;
  *h_len = len;
  return HLB_OK;
}

hlb_status hlb_batch_flux_history(hlb_batch* b, int i, double* h_out, int max_len, int* h_len) {
  if (!batch_ok(b, i)) return HLB_EINVAL;
  return hlb_flux_history(&b->dom[i], h_out, max_len, h_len);
}

hlb_status hlb_batch_stop(hlb_batch* b, int i) {
  if (!batch_ok(b, i)) return HLB_EINVAL;
  if (!b->active[i]) return HLB_OK;
  b->active[i] = 0;
  const int zero = 0;
  if (cudaMemcpyAsync(b->d_active + i, &zero, sizeof(int), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return HLB_ECUDA;
  return HLB_OK;
}

hlb_status hlb_batch_checkpoint_save(hlb_batch* b, int i, void* h_buf, size_t cap, size_t* h_len) {
  if (!batch_ok(b, i)) return HLB_EINVAL;
  return ckpt_save(&b->dom[i], h_buf, cap, h_len);
}

hlb_status hlb_batch_checkpoint_load(hlb_batch* b, int i, const void* h_buf, size_t len) {
  if (!batch_ok(b, i)) return HLB_EINVAL;
  // the domain rejoins the batch at the batch's current buffer parity
  hlb_status st = ckpt_load(&b->dom[i], h_buf, len, b->parity);
  if (st != HLB_OK) return st;
  k_lag_from_state<<<1, 32, 0, b->stream>>>(b->dom[i].state, b->d_lag + i);
  if (cudaGetLastError() != cudaSuccess) return HLB_ECUDA;
  b->active[i] = 1;
  batch_drop_graph(b);
  return upload_tables(b);  // T_bottom in the descriptors, the active flag
}

hlb_status hlb_batch_destroy(hlb_batch* b) {
  if (!b) return HLB_EINVAL;
  batch_drop_graph(b);
  for (auto& d : b->dom) drop_graph(&d);
  delete b;
  return HLB_OK;
}

// ------------------------------------------------------------- autotuning
namespace {

}  // namespace

hlb_status hlb_autotune(hlb_domain* d, int steps_per_variant, int* chosen, float* h_ms, int max_out) {
  if (!d || steps_per_variant < 1 || !chosen) return HLB_EINVAL;
  if (!d->fields_set || d->host_flags) return HLB_ESTATE;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HLB_ECUDA;
  float best = 1e30f;
  int best_v = 0;
  hlb_status st = HLB_OK;
  for (int v = 0; v < NV_ALL && st == HLB_OK; ++v) {
    if (!variant_ok(d, v)) {
      if (h_ms && v < max_out) h_ms[v] = 1e30f;  // not available for this width, scheme or N
      continue;
    }
    set_variant_grids(d, v);
    drop_graph(d);
    st = launch_step(d);  // one untimed step per variant (first-launch costs)
    cudaEventRecord(e0, d->stream);
    for (int k = 0; k < steps_per_variant && st == HLB_OK; ++k) st = launch_step(d);
    cudaEventRecord(e1, d->stream);
    float ms = 0.f;
    if (st == HLB_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = HLB_ECUDA;
    ms /= (float)steps_per_variant;
    if (h_ms && v < max_out) h_ms[v] = ms;
    if (ms < best) {
      best = ms;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  set_variant_grids(d, best_v);
  drop_graph(d);
  *chosen = best_v;
  return st;
}

hlb_status hlb_batch_autotune(hlb_batch* b, int steps_per_variant, int* chosen, float* h_ms, int max_out) {
  if (!b || steps_per_variant < 1 || !chosen) return HLB_EINVAL;
  for (int i = 0; i < b->n; ++i)
    if (!b->dom[i].fields_set) return HLB_ESTATE;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HLB_ECUDA;
  float best = 1e30f;
  int best_v = 0;
  hlb_status st = HLB_OK;
  for (int v = 0; v < NV_ALL && st == HLB_OK; ++v) {
    if (!batch_variant_ok(b, v)) {
      if (h_ms && v < max_out) h_ms[v] = 1e30f;  // not available for these widths or this N
      continue;
    }
    st = set_batch_variant(b, v);
    if (st != HLB_OK) break;
    st = batch_launch(b, nullptr, nullptr);  // one untimed step per variant (first-launch costs)
    if (st != HLB_OK) break;
    if (st == HLB_OK) st = lane_join(b);
    cudaEventRecord(e0, b->stream);
    for (int k = 0; k < steps_per_variant && st == HLB_OK; ++k) st = batch_launch(b, nullptr, nullptr);
    if (st == HLB_OK) st = lane_join(b);
    cudaEventRecord(e1, b->stream);
    float ms = 0.f;
    if (st == HLB_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = HLB_ECUDA;
    ms /= (float)steps_per_variant;
    if (h_ms && v < max_out) h_ms[v] = ms;
    if (ms < best) {
      best = ms;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const hlb_status st2 = set_batch_variant(b, best_v);
  *chosen = best_v;
  return st != HLB_OK ? st : st2;
}

hlb_status hlb_set_tile_variant(hlb_domain* d, int v) {
  if (!d || v < 0 || v >= NV_ALL) return HLB_EINVAL;
  if (!variant_ok(d, v)) return HLB_EINVAL;
  set_variant_grids(d, v);
  drop_graph(d);
  return HLB_OK;
}

hlb_status hlb_batch_set_tile_variant(hlb_batch* b, int v) {
  if (!b || v < 0 || v >= NV_ALL) return HLB_EINVAL;
  return set_batch_variant(b, v);
}

int hlb_tile_variants(int* h_tile_w, int* h_tile_h, int* h_threads, int max_out) {
  for (int v = 0; v < NV_ALL && v < max_out; ++v) {
    // split step: the flow tile (64 columns, fluid rows, threads); fused tiled:
    // the 52-column tile; row-marching: full width (0), segment height, one
    // thread per column (0)
    if (is_split(v)) {
      if (h_tile_w) h_tile_w[v] = FL_TX;
      if (h_tile_h) h_tile_h[v] = FLOWS[v].ty;
      if (h_threads) h_threads[v] = FLOWS[v].nth;
    } else if (is_march(v)) {
      if (h_tile_w) h_tile_w[v] = 0;
      if (h_tile_h) h_tile_h[v] = march_seg(v);
      if (h_threads) h_threads[v] = 0;
    } else {
      if (h_tile_w) h_tile_w[v] = TILE_X;
      if (h_tile_h) h_tile_h[v] = VARIANTS[tiled_index(v)].ty;
      if (h_threads) h_threads[v] = VARIANTS[tiled_index(v)].nth;
    }
  }
  return NV_ALL;
}

int hlb_variant_kind(int v) {
  if (v < 0 || v >= NV_ALL) return -1;
  return is_split(v) ? HLB_KIND_SPLIT : (is_march(v) ? HLB_KIND_MARCH : HLB_KIND_FUSED);
}

int hlb_variant_energy_rows(int v) {
  if (v < 0 || v >= NV_ALL || !is_split(v)) return -1;
  return FLOWS[v].ewalk ? FLOWS[v].ep : 0;
}

const char* hlb_strerror(hlb_status s) {
  switch (s) {
    case HLB_OK: return "ok";
    case HLB_EINVAL: return "invalid argument";
    case HLB_ECUDA: return "CUDA runtime error";
    case HLB_EUNSTABLE: return "device error word set (non-finite value or psi^2 < 0)";
    case HLB_ETIMEOUT: return "bounded device wait timed out";
    case HLB_ESTATE: return "call not valid in the current state";
  }
  return "unknown status";
}

}  // extern "C"

// ===================================================================
// hlb_step_static: one coupled step whose scratch memory is a static device
// array inside this library, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where no allocator is available or allowed --
// a solver embedded as a plug-in in a host application that owns every device
// allocation through its own pool, or a process whose device memory is fully
// reserved up front.  Such a caller can
// still hand over its own state buffers (inputs and outputs), but cannot give
// the library a workspace for the per-block FP64 partial sums, the device-side
// diagnostics record and the wetting table.  This entry point takes those from
// `g_scratch` below instead, and calls no cudaMalloc, cudaFree or allocating
// library routine.
//
// The scratch array is HLB_STATIC_SCRATCH_BYTES (1 MiB) of device memory that
// every GPU which loads the library holds until the process exits.  Every call
// shares it and it keeps the last call's contents; the diagnostics record is
// cleared at the start of each call and the partial sums are fully rewritten by
// each step, so no call sees stale values.  Calls that overlap on the GPU (two
// streams, or two host threads) race on the shared array.  Each call reads the
// step's diagnostics back to the host and synchronises its stream.

namespace {

constexpr size_t STATE_BYTES = 256;
constexpr size_t GW_BYTES = (size_t)HLB_STATIC_MAX_NX * sizeof(float);
constexpr size_t PART_BYTES = HLB_STATIC_SCRATCH_BYTES - STATE_BYTES - GW_BYTES;
constexpr long long MAX_BLOCKS = (long long)(PART_BYTES / (NPART * sizeof(double)));
static_assert(sizeof(DevState) <= STATE_BYTES, "device record does not fit its slot");

// The scratch itself: [DevState | G_w table | per-block partials].
static __device__ __align__(256) unsigned char g_scratch[HLB_STATIC_SCRATCH_BYTES];

// In host code the name g_scratch is only a stand-in, not a device address;
// the real address comes from cudaGetSymbolAddress with the device current.

struct StaticSites {
  int n;
  hlb_site s[HLB_STATIC_MAX_SITES];
};

// Clear the diagnostics record and set this step's lagged inputs; build the
// wetting table (Section 4.2, Fig. 6b) from the sites.
__global__ void k_static_prepare(DevState* st, float* Gw, int nx, double Gw0, StaticSites sites, double rho_ave,
                                 double U) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    st->rho_ave = rho_ave;
    st->rho_ave_prev = rho_ave;
    st->U = U > 0.0 ? U : 0.0;
    st->Uc = st->U / (1.0 + st->U);
    st->step = 0;
    st->mass = st->energy = st->q_bottom = st->q_top = st->q_interface = st->u_top = 0.0;
    st->q_sum = 0.0;
    st->q_count = 0;
    st->error_flags = 0;
    st->hist_len = 0;
  }
  for (int x = t; x < nx; x += gridDim.x * blockDim.x) {
    double g = Gw0;
    for (int k = 0; k < sites.n; ++k) {
      const double half = 0.5 * sites.s[k].width;
      double d = fabs((double)x - sites.s[k].x_center);
      d = fmin(d, (double)nx - d);
      if (d <= half) g = fmin(g, sites.s[k].gw_min + (Gw0 - sites.s[k].gw_min) * d / half);
    }
    Gw[x] = (float)g;
  }
}

// On every call, with the caller's device current: resolve the address of
// g_scratch (cheap, allocates nothing) and allow the step kernel its dynamic
// shared memory.  Nothing is cached, so a device reset or a new primary
// context between calls cannot leave a stale address behind.
hlb_status setup_device(void** addr) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return HLB_ECUDA;
  if (cudaFuncSetAttribute(VARIANTS[0].single_fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)VARIANTS[0].smem) != cudaSuccess)
    return HLB_ECUDA;
  *addr = p;
  return HLB_OK;
}

}  // namespace

extern "C" hlb_status hlb_step_static(const hlb_params* p, int n_sites, const hlb_site* h_sites,
                                      const float* d_f_in, float* d_f_out, const float* d_T_in, float* d_T_out,
                                      const float* d_ftop_in, float* d_ftop_out, double rho_ave, double U,
                                      hlb_diag_record* h_out, void* stream) {
  if (!p || !d_f_in || !d_f_out || !d_T_in || !d_T_out || !h_out) return HLB_EINVAL;
  if (n_sites < 0 || n_sites > HLB_STATIC_MAX_SITES || (n_sites > 0 && !h_sites)) return HLB_EINVAL;
  if (hlb_workspace_bytes(p) == 0) return HLB_EINVAL;  // the same parameter checks as hlb_init
  if (resolved_nsub(p) != 1) return HLB_EINVAL;         // sub-steps need workspace scratch
  if (p->top_bc == HLB_TOP_CONVECTIVE && (!d_ftop_in || !d_ftop_out)) return HLB_EINVAL;
  if (p->nx > HLB_STATIC_MAX_NX) return HLB_EINVAL;
  const long long nblk = (long long)((p->nx + TILE_X - 1) / TILE_X) * ((p->ny + TILE_Y - 1) / TILE_Y);
  if (nblk > MAX_BLOCKS) return HLB_EINVAL;  // lattice larger than the static scratch serves
  if (!(rho_ave > 0.0) || !isfinite(U)) return HLB_EINVAL;

  void* base = nullptr;
  const hlb_status st0 = setup_device(&base);
  if (st0 != HLB_OK) return st0;
  unsigned char* scratch = (unsigned char*)base;
  DevState* state = (DevState*)scratch;
  float* Gw = (float*)(scratch + STATE_BYTES);
  double* partials = (double*)(scratch + STATE_BYTES + GW_BYTES);
  cudaStream_t s = (cudaStream_t)stream;

  // parameters, resolved as hlb_init resolves them (no allocation: host stack only)
  hlb_params q = *p;
  q.n_sub = 1;  // checked above: n_sub is 1, or 0 resolving to 1
  double Tc = 0.0;
  if (!(q.rho_l > 0 && q.rho_v > 0)) {
    if (hlb_eos_coexistence(p, &Tc, &q.rho_l, &q.rho_v, nullptr) != HLB_OK) return HLB_EINVAL;
  } else if (hlb_eos_coexistence(p, &Tc, nullptr, nullptr, nullptr) != HLB_OK) {
    Tc = (q.a / q.b) * (0.0778 / 0.45724) / q.R;
  }
  if (!(q.rho_w > 0)) q.rho_w = 3.0 * q.rho_l;
  if (!(q.cv_w > 0)) q.cv_w = q.cv;
  if (!(q.lambda_w > 0)) q.lambda_w = 3.0 * q.rho_l * q.cv * q.k;
  const double kappa = 0.37464 + 1.54226 * q.omega - 0.26992 * q.omega * q.omega;

  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.nx = q.nx;
  a.ny = q.ny;
  a.W = q.wall_rows;
  a.top_bc = q.top_bc;
  a.eos_T_fixed = q.eos_T_fixed;
  a.plane = (long long)q.nx * q.ny;
  a.R = (float)q.R;
  a.a = (float)q.a;
  a.b = (float)q.b;
  a.kappa = (float)kappa;
  a.invTc = (float)(1.0 / Tc);
  a.Ts = (float)(q.Ts_over_Tc * Tc);
  a.G = (float)q.G;
  a.g_y = (float)q.g_y;
  a.sig_e = (float)((1.0 - 0.5 * q.s_e) * q.sigma_coef * q.sigma / (1.0 / q.s_e - 0.5));
  a.sig_z = (float)((1.0 - 0.5 * q.s_zeta) * q.sigma_coef * q.sigma / (1.0 / q.s_zeta - 0.5));
  a.s_e = (float)q.s_e;
  a.s_z = (float)q.s_zeta;
  a.s_j = (float)q.s_j;
  a.s_q = (float)q.s_q;
  a.tau_l = (float)q.tau_l;
  a.tau_v = (float)q.tau_v;
  a.rho_v = (float)q.rho_v;
  a.dtau_drho = (float)((q.tau_l - q.tau_v) / (q.rho_l - q.rho_v));
  a.rho_ref = (float)(q.storage == HLB_STORE_DEVIATION ? q.rho_v : 0.0);
  a.rho_mid = (float)(0.5 * (q.rho_l + q.rho_v));
  a.cvk = (float)(q.cv * q.k);
  a.cv = (float)q.cv;
  a.rcv_w = (float)(q.rho_w * q.cv_w);
  a.inv_rcv_w = (float)(1.0 / (q.rho_w * q.cv_w));
  a.lambda_w = (float)q.lambda_w;
  a.lambda_top = (float)(q.lambda_top > 0 ? q.lambda_top : q.lambda_w);
  a.bottom_flux = q.bottom_bc == HLB_BOTTOM_FLUX ? 1 : 0;
  a.q_in = (float)q.q_in;
  a.dt = (float)(1.0 / q.n_sub);
  a.iso = q.diffusion == HLB_DIFF_ISO ? 1 : 0;
  a.kd = (float)q.k;
  a.kd_w = (float)(q.lambda_w / (q.rho_w * q.cv_w));
  a.T_bottom = (float)q.T_bottom;
  a.T_top = (float)q.T_top;
  a.f_in = d_f_in;
  a.f_out = d_f_out;
  a.T_in = d_T_in;
  a.T_out = d_T_out;
  a.Gw = Gw;
  a.ftop_in = d_ftop_in;
  a.ftop_out = d_ftop_out;
  a.partials = partials;
  a.state = state;

  StaticSites sites;
  memset(&sites, 0, sizeof(sites));
  sites.n = n_sites;
  for (int k = 0; k < n_sites; ++k) {
    if (!(h_sites[k].width > 0)) return HLB_EINVAL;
    sites.s[k] = h_sites[k];
  }
  const int fluid_rows = q.ny - q.wall_rows - (q.top_bc == HLB_TOP_WALL ? 1 : 0);
  const double n_fluid = (double)fluid_rows * q.nx;

  k_static_prepare<<<(q.nx + 255) / 256, 256, 0, s>>>(state, Gw, q.nx, q.Gw0, sites, rho_ave, U);
  VARIANTS[0].launch_single(grid_of(q.nx, q.ny, q.wall_rows, q.top_bc, FIRST_TILED), VARIANTS[0].smem, s, a);
  k_reduce<<<1, 256, 0, s>>>(partials, (int)nblk, state, 1.0 / n_fluid, 1.0 / (double)q.nx, nullptr, 0);
  if (cudaGetLastError() != cudaSuccess) return HLB_ECUDA;

  DevState out;
  if (cudaMemcpyAsync(&out, state, sizeof(out), cudaMemcpyDeviceToHost, s) != cudaSuccess) return HLB_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return HLB_ECUDA;
  h_out->step = out.step;
  h_out->mass = out.mass;
  h_out->energy = out.energy;
  h_out->q_bottom = out.q_bottom;
  h_out->q_top = out.q_top;
  h_out->q_interface = out.q_interface;
  h_out->rho_ave = out.rho_ave;
  h_out->u_top = out.u_top;
  h_out->q_bottom_timeavg = out.q_bottom;
  h_out->vapour_coverage = out.vcov;
  h_out->vapour_coverage_timeavg = out.vcov;
  h_out->error_flags = out.error_flags;
  if (out.error_flags & ERR_TIMEOUT) return HLB_ETIMEOUT;
  return out.error_flags ? HLB_EUNSTABLE : HLB_OK;
}
