/*
 * hlb.h - C ABI of the GB300 (sm_103a) hybrid thermal lattice Boltzmann
 * phase-change step of Hu & Liu, "Study of boiling heat transfer on the wall
 * with an improved hybrid lattice Boltzmann model" (arXiv 1812.10375).
 *
 * One step of a domain is: D2Q9 MRT pseudo-potential collide-and-stream
 * (Section 2.1, Eqs. 1-10), Peng-Robinson EOS (Section 3.1, Eq. 28), the energy
 * equation (Eq. 17) advanced by N RK4 sub-steps of dt/N (Eqs. 18, 27) and
 * finite-volume diffusion with harmonic face conductivities (Eqs. 22-26),
 * halfway bounce-back walls, a conjugate heater and open tops (Sections 3.3,
 * 4.2), and the wettability nucleation sites of Section 4.2 (Fig. 6b).
 *
 * Conventions shared by every entry point:
 *  - Lattice arrays are row-major [y][x] with x fastest, nx*ny elements, FP32.
 *    Row 0 is the bottom (heater) row; x is periodic.
 *  - Pointers named d_* are CUDA device pointers; h_* are host pointers.
 *  - The caller owns every buffer and the stream.  The library never allocates
 *    device memory: it works inside the workspace the caller passes to
 *    hlb_init / hlb_batch_init, which must stay valid until hlb_destroy.
 *  - Host pointers are read or written only during the call.
 *  - Every call returns an hlb_status and never throws or aborts.  Kernels are
 *    launched asynchronously on the handle's stream; hlb_diag and the flux
 *    history and checkpoint calls synchronise that stream.
 *  - Device-side problems set a sticky error word (bit 0: non-finite value,
 *    bit 1: psi^2 < 0 outside the EOS range, bit 2: a bounded device wait gave
 *    up; no kernel of this library waits on another block, so bit 2 is
 *    reserved and never set).
 *    hlb_diag reports it; once it is set, hlb_step returns HLB_ESTATE.
 *  - A handle is not thread-safe: use it from one host thread at a time.
 *  - `stream` arguments are cudaStream_t values passed as void* (NULL = the
 *    legacy default stream).
 */
#ifndef HLB_H
#define HLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HLB_OK = 0,
  HLB_EINVAL = -1,     /* bad argument or parameter set                  */
  HLB_ECUDA = -2,      /* a CUDA runtime call failed                      */
  HLB_EUNSTABLE = -3,  /* the device error word reports non-finite / psi  */
  HLB_ETIMEOUT = -4,   /* a bounded device wait gave up (reserved)        */
  HLB_ESTATE = -5      /* call not valid in the handle's current state    */
} hlb_status;

/* Top boundary kinds (Sections 3.2, 3.3, 4.2). */
enum { HLB_TOP_WALL = 0, HLB_TOP_CONST_RHO = 1, HLB_TOP_CONVECTIVE = 2 };

/* Distribution storage (precision pattern): deviations f_i - w_i rho_ref (default)
 * or the plain populations. */
enum { HLB_STORE_DEVIATION = 0, HLB_STORE_PLAIN = 1 };

/* Diffusion term of the energy equation (Eq. 17): the finite-volume form with
 * harmonic face conductivities (Eqs. 22-26, the paper's scheme, default), or
 * the isotropic central form lambda lap(T) + grad(lambda) . grad(T) with the
 * Laplacian of Eq. (20) and the gradients of Eq. (19) (Eq. 21, the scheme the
 * paper shows to violate energy conservation across conductivity jumps,
 * Section 3.2).  The isotropic form runs in the single-domain tiled kernel only;
 * batches and the row-marching kernel reject it. */
enum { HLB_DIFF_FV = 0, HLB_DIFF_ISO = 1 };

/* Bottom thermal boundary: row 0 held at T_bottom (default), or heated by an
 * imposed flux q_in (heat per unit time and unit length entering row 0
 * through its bottom face, Section 3.3); row 0 then evolves like the other
 * heater rows.  q_bottom in the diagnostics is always the flux through the
 * face between rows 0 and 1. */
enum { HLB_BOTTOM_DIRICHLET = 0, HLB_BOTTOM_FLUX = 1 };

/*
 * Model and geometry parameters, all in lattice units (dx = dt = 1, Section 3.1).
 * hlb_params_default fills the paper's values; fields marked "<= 0: default"
 * are derived at init from the coexistence densities.
 */
typedef struct {
  int nx, ny;          /* lattice size; nx >= 4, ny >= 6                            */
  int wall_rows;       /* rows y < wall_rows are solid (>= 1); row 0 has Dirichlet T */
  int top_bc;          /* HLB_TOP_*; HLB_TOP_WALL makes row ny-1 a solid Dirichlet row */
  int eos_T_fixed;     /* 1: the EOS uses Ts everywhere (Section 3.2)               */
  int n_sub;           /* N of Eq. (27), 1..64, or 0: hlb_stable_substeps (1 for the
                          paper's parameters).  N > 1 holds rho^n and u^n over the
                          sub-steps and runs with HLB_DIFF_FV, for single domains
                          and batches (a batch shares one N); the isotropic scheme
                          and hlb_step_static take N = 1 only                     */
  int storage;         /* HLB_STORE_DEVIATION | HLB_STORE_PLAIN                      */
  double a, b, R, omega, Ts_over_Tc;   /* Eq. (28): 3/49, 2/21, 1, 0.344, 0.86        */
  double G, sigma, sigma_coef;         /* Eqs. (6)-(8): -1, 0.107, 12                 */
  double s_rho, s_e, s_zeta, s_j, s_q; /* Eq. (3) rates not printed: 1, .8, .8, 1, 1.1 */
  double tau_l, tau_v;                 /* tau_nu at rho_l / rho_v: 0.8, 1.0 (Sec. 3.1) */
  double cv, k;                        /* Section 3.1: 6, 0.1 (lambda = rho cv k)     */
  double rho_w, cv_w, lambda_w;        /* solid; <= 0: default 3 rho_l, cv, 3 rho_l cv k */
  double g_y;                          /* gravity (Eq. 9), e.g. -3e-5                 */
  double Gw0;                          /* wall wetting strength (Eq. 10), 0.3         */
  double T_bottom, T_top;              /* Dirichlet T of row 0 / of row ny-1 (top wall) */
  double rho_l, rho_v;                 /* coexistence densities at Ts; <= 0: Maxwell  */
  int diffusion;                       /* HLB_DIFF_FV (default) | HLB_DIFF_ISO         */
  double lambda_top;                   /* conductivity of a top wall row; <= 0: lambda_w
                                          (Section 3.2: each wall conducts like the phase
                                          next to it)                                   */
  int bottom_bc;                       /* HLB_BOTTOM_DIRICHLET (default) | HLB_BOTTOM_FLUX */
  double q_in;                         /* imposed heat flux into row 0 (HLB_BOTTOM_FLUX) */
} hlb_params;

/* One nucleation site: a linear drop of G_w from Gw0 to gw_min at x_center over
 * width/2 on either side (Section 4.2, Fig. 6b). */
typedef struct { double x_center, width, gw_min; } hlb_site;

/* FP64 diagnostics of the last completed step (Eq. 9 rho_ave; Section 4.3 wall
 * heat flux).  q_* are RK-weighted conductive fluxes through a face over the
 * step, averaged over x (heat per unit time and unit length). */
typedef struct {
  long long step;         /* completed steps                                    */
  double mass;            /* sum of rho over fluid nodes                        */
  double energy;          /* sum of rho cv T over all nodes (T after the step)  */
  double q_bottom;        /* into row 1 through the bottom Dirichlet face       */
  double q_top;           /* out of row ny-2 through the top Dirichlet face     */
  double q_interface;     /* through the solid -> fluid face                     */
  double rho_ave;         /* mean fluid density, used by the next step (Eq. 9)  */
  double u_top;           /* mean u_y of row ny-2                                */
  double q_bottom_timeavg;/* running mean of q_bottom since the last reset      */
  int error_flags;        /* sticky device error word                            */
  double vapour_coverage; /* vapour fraction (rho < (rho_l + rho_v)/2) of the
                             first fluid row above the wall                      */
  double vapour_coverage_timeavg; /* its running mean since the last reset      */
} hlb_diag_record;

typedef struct hlb_domain hlb_domain;
typedef struct hlb_batch hlb_batch;

/* Fill the paper's parameter values (Section 3.1) for an nx x ny lattice. */
void hlb_params_default(hlb_params* p, int nx, int ny);

/* Host-only: the N of Eq. (27) that n_sub = 0 selects, the smallest N for which
 * one RK4 sub-step of dt/N is stable for the finite-volume conduction operator
 * (Section 2.2 leaves N to stability).  The operator's eigenvalues are real
 * and within [-16 D, 0], D the largest of k (the fluid) and
 * lambda_w / (rho_w cv_w) (the heater), by Gershgorin's theorem with harmonic
 * face conductivities at most twice a cell's own.  RK4 is stable on the
 * negative real axis down to -2.785, so N = ceil(16 D / 2.785).  Advection and
 * the latent-heat term are not part of the bound.  Returns 0 on invalid
 * parameters; a parameter set with n_sub = 0 is refused when this N exceeds 64. */
int hlb_stable_substeps(const hlb_params* p);

/* Host-only: Tc (from a, b, R), and the Maxwell equal-area coexistence
 * densities at T = Ts_over_Tc * Tc (Section 3.1), plus the latent heat of
 * Eq. (14) per unit mass.  Any out pointer may be NULL.  HLB_EINVAL when the
 * temperature has no two-phase region. */
hlb_status hlb_eos_coexistence(const hlb_params* p, double* Tc, double* rho_l, double* rho_v,
                               double* h_fg);

/* Device bytes one domain needs (fields double-buffered, per-block FP64 partials,
 * site table, flux history, the rho^n, u^n and scratch T planes of the split
 * step; for N > 1 also the fused kernels' sub-step partials).  0 on invalid parameters, which include lattices
 * whose nine population planes would exceed 2^31 floats (about 238 million
 * cells, e.g. 15,000 x 15,000 fits, 16,384 x 16,384 does not). */
size_t hlb_workspace_bytes(const hlb_params* p);

/* Create a domain inside the caller's device workspace (>= hlb_workspace_bytes
 * bytes, 256-byte aligned).  Parameters are copied; unset derived values are
 * filled.  The initial wetting table is the constant Gw0; fields are unset
 * until hlb_set_fields.  *out is owned by the library until hlb_destroy. */
hlb_status hlb_init(hlb_domain** out, const hlb_params* p, void* d_workspace, size_t workspace_bytes,
                    void* stream);

/* Initial state: rho and T (device, nx*ny FP32 each).  Populations become the
 * rest equilibrium w_i rho; Dirichlet rows take their wall value; rho_ave is the
 * fluid mean of rho; the step counter and time averages reset. */
hlb_status hlb_set_fields(hlb_domain* d, const float* d_rho, const float* d_T);

/* Dirichlet wall temperature of row 0 (the heater bottom, Section 4.2; the
 * hot wall of Section 3.2).  Takes effect from the next step. */
hlb_status hlb_set_wall(hlb_domain* d, double T_bottom);

/* Wetting table from nucleation sites (Section 4.2): G_w(x) = Gw0 except inside
 * a site, where it drops linearly to gw_min at the centre (periodic in x; the
 * lowest value wins where sites overlap).  n = 0 restores the uniform wall. */
hlb_status hlb_set_nucleation_sites(hlb_domain* d, int n, const hlb_site* h_sites);

/* Advance nsteps coupled steps (asynchronous on the handle's stream).
 * Repeated calls reuse a captured CUDA graph of 16 steps.  A step of the split
 * form (the default for HLB_DIFF_FV) is a flow kernel, N energy sub-step
 * kernels and an FP64 reduction kernel; a step of a fused variant is the fused
 * step kernel and the reduction (see the autotuning section). */
hlb_status hlb_step(hlb_domain* d, int nsteps);

/* Fields after the last step: rho^n, u^n (the step's pre-collision moments,
 * Eq. 5) and T^{n+1}.  Any pointer may be NULL.  Before the first step: the
 * initial rho, u = 0 and the initial T. */
hlb_status hlb_read(hlb_domain* d, float* d_rho, float* d_ux, float* d_uy, float* d_T);

/* Copy the FP64 diagnostics of the last step to the host (synchronises the
 * stream).  Returns HLB_EUNSTABLE if the device error word is set (the record is
 * still written). */
hlb_status hlb_diag(hlb_domain* d, hlb_diag_record* h_out);

/* Copy the per-step wall heat flux q_bottom (FP64, one entry per step since
 * hlb_set_fields, at most 65536 entries) into h_out[0..max_len); *h_len
 * receives the number written.  Synchronises the stream. */
hlb_status hlb_flux_history(hlb_domain* d, double* h_out, int max_len, int* h_len);

/* Restart the running time averages (q_bottom, vapour coverage) at the next step. */
hlb_status hlb_reset_timeavg(hlb_domain* d);

/* Release the handle (the workspace stays the caller's). */
hlb_status hlb_destroy(hlb_domain* d);

/* ------------------------------------------------------ checkpoint / resume
 * The paper has no counterpart; long boiling runs (Section 4.3 averages the wall
 * flux over tens of thousands of steps) need to survive a lost process.  A
 * checkpoint is a byte image, in host memory, of everything one domain carries
 * from a step to the next, taken at a step boundary:
 *   a 512-byte header (magic "HLBCKPT1", format version, lattice size, wall
 *   rows, top and bottom boundary kinds, storage form and its reference
 *   density, T_bottom, the step counter and the device diagnostics record with
 *   the lagged rho_ave and outlet velocity of Eq. 9 and the running sums),
 *   then FP32 arrays: the nine population planes (nx*ny each, the storage form
 *   of the domain), T^{n+1}, T^n, the convective-outlet memory (3*nx), the
 *   wetting table (nx), then, 8-byte aligned, the hist_len FP64 entries of the
 *   per-step wall-flux history.
 * Stepping a domain restored from a checkpoint gives bit-for-bit the states the
 * saved domain would have reached (same library build and variant).
 *
 * hlb_checkpoint_bytes: the largest checkpoint of a domain with parameters p
 * (full flux history); 0 on invalid parameters.
 * hlb_checkpoint_save: writes the checkpoint of the state after the last step
 * into h_buf[0..cap) and its length into *h_len (synchronises the stream).
 * HLB_ESTATE before hlb_set_fields; HLB_EINVAL if cap is too small.
 * hlb_checkpoint_load: replaces the domain's state by the checkpoint in
 * h_buf[0..len) (synchronises).  The lattice size, wall rows, boundary kinds and
 * storage form (with its reference density) must equal the domain's, else
 * HLB_EINVAL and the domain is unchanged; the other model parameters are the
 * domain's own.  T_bottom and the wetting table are restored from the
 * checkpoint.  A checkpoint whose error word is set restores that word too
 * (later steps then return HLB_ESTATE).
 * hlb_batch_checkpoint_save / _load: the same for domain i of a batch; loading
 * makes domain i active again. */
size_t hlb_checkpoint_bytes(const hlb_params* p);
hlb_status hlb_checkpoint_save(hlb_domain* d, void* h_buf, size_t cap, size_t* h_len);
hlb_status hlb_checkpoint_load(hlb_domain* d, const void* h_buf, size_t len);

/* ------------------------------------------------------------------ batch
 * A boiling-curve sweep: n independent domains (each with its own size,
 * superheat and sites; one model parameter set, N of Eq. 27 included)
 * advanced together.  In the split form (default) one step is a single launch
 * of the flow kernel whose blocks cover the flow tiles of every active domain
 * (a descriptor table maps block -> domain, tile), N launches of the energy
 * sub-step kernel over every domain's energy tiles, and one FP64 reduction
 * launch with one CTA per domain; a fused variant replaces the first two by
 * one launch of the fused step kernel (N = 1 only).  Repeated hlb_batch_step
 * calls replay a captured CUDA graph of 16 such steps. */

/* Device bytes for n domains with parameters p[0..n-1]; 0 if any is invalid. */
size_t hlb_batch_workspace_bytes(int n, const hlb_params* p);

/* Create a batch inside the caller's workspace (256-byte aligned).  Each
 * domain behaves as one made by hlb_init. */
hlb_status hlb_batch_init(hlb_batch** out, int n, const hlb_params* p, void* d_workspace, size_t workspace_bytes,
                          void* stream);

/* Per-domain set-up, as hlb_set_fields / hlb_set_wall / hlb_set_nucleation_sites
 * for domain i (0 <= i < n).  hlb_batch_set_fields may be called at any time: it
 * restarts domain i from the given fields (step counter, time average and flux
 * history reset) and makes it active again, so a slot can be reused for a new
 * sweep point. */
hlb_status hlb_batch_set_fields(hlb_batch* b, int i, const float* d_rho, const float* d_T);
hlb_status hlb_batch_set_wall(hlb_batch* b, int i, double T_bottom);
hlb_status hlb_batch_set_nucleation_sites(hlb_batch* b, int i, int n, const hlb_site* h_sites);

/* Advance every active domain by nsteps (asynchronous). */
hlb_status hlb_batch_step(hlb_batch* b, int nsteps);

/* One batch step launched directly (no graph), with the caller's CUDA events
 * (cudaEvent_t as void*, either may be NULL) recorded on the batch stream
 * immediately before and after the step kernels (the fused step kernel, or
 * the flow and energy kernels of a split step), so that their duration can be
 * measured apart from the reduction. */
hlb_status hlb_batch_step_profiled(hlb_batch* b, void* ev_before, void* ev_after);

/* As hlb_batch_step_profiled, with one more event (may be NULL) recorded
 * between the flow kernel and the energy kernels of a split step (not
 * recorded by a fused variant, nor in two lanes), so that each kernel can be
 * timed. */
hlb_status hlb_batch_step_phases(hlb_batch* b, void* ev_before, void* ev_flow, void* ev_after);

/* Lanes of the split step (lanes = 1 or 2; 1 after hlb_batch_init).  With 2,
 * the domains are cut into two contiguous groups of about equal cell count;
 * the second group's launches go to a stream of the library's own, and its
 * flow kernel of a step waits only for the first group's, so that the
 * first group's energy kernels run beside the second group's flow kernel and
 * the second's energy kernels beside the first's next flow kernel.  Results
 * are those of one lane bit for bit (the groups' domains are independent).
 * Every batch call returns with the second stream joined into the batch
 * stream, so the caller still sees one stream.  HLB_EINVAL for another lane
 * count; a batch of one domain or a fused variant runs in one lane. */
hlb_status hlb_batch_set_lanes(hlb_batch* b, int lanes);

/* As hlb_read / hlb_diag for domain i. */
hlb_status hlb_batch_read(hlb_batch* b, int i, float* d_rho, float* d_ux, float* d_uy, float* d_T);
hlb_status hlb_batch_diag(hlb_batch* b, int i, hlb_diag_record* h_out);

/* Copy domain i's per-step wall heat flux q_bottom (FP64, one entry per step
 * since hlb_batch_set_fields, at most 65536 entries) into h_out[0..max_len);
 * *h_len receives the number written.  Synchronises the stream. */
hlb_status hlb_batch_flux_history(hlb_batch* b, int i, double* h_out, int max_len, int* h_len);

/* Stop domain i: later batch steps skip it and its state stays readable
 * (early stop of a sweep point). */
hlb_status hlb_batch_stop(hlb_batch* b, int i);

/* Checkpoint of domain i (see hlb_checkpoint_save / hlb_checkpoint_load). */
hlb_status hlb_batch_checkpoint_save(hlb_batch* b, int i, void* h_buf, size_t cap, size_t* h_len);
hlb_status hlb_batch_checkpoint_load(hlb_batch* b, int i, const void* h_buf, size_t len);

hlb_status hlb_batch_destroy(hlb_batch* b);

/* ------------------------------------------------------------- autotuning
 * The step is compiled in three kinds (hlb_variant_kind):
 *  - HLB_KIND_SPLIT: a flow kernel over tiles of 64 columns by a few fluid-row
 *    heights, then N energy sub-step kernels: a row-walking kernel over strips
 *    of 56 columns and segments of 96, 64 or 32 rows, or a tiled one over
 *    56 x 24 tiles (finite-volume scheme; the default for it);
 *  - HLB_KIND_FUSED: one fused step kernel over 52-column tiles of a few
 *    heights, with 256 or 512 threads per CTA (the default for the isotropic
 *    scheme, which only this kind runs);
 *  - HLB_KIND_MARCH: one fused kernel per full-width segment of 32, 48 or 64
 *    rows, one thread per column, for lattices up to 512 columns and the
 *    finite-volume scheme only (a batch launches one kernel per row stride).
 * hlb_tile_variants lists them in that order (returns their count; arrays may
 * be NULL): a split variant reports its flow tile's width, height and threads,
 * a fused tiled one its tile's, a row-marching one width 0, its segment height
 * and 0 threads.  hlb_variant_kind(v) returns the kind of variant v, or -1;
 * hlb_variant_energy_rows(v) the segment height of a split variant's
 * row-walking energy kernel, 0 for a split variant with the tiled energy
 * kernel, -1 for the other kinds or v out of range.  hlb_autotune / hlb_batch_autotune run one untimed and
 * then steps_per_variant timed steps of every variant available to the
 * handle on its own state (others report 1e30 ms), keep the fastest for later
 * steps and report its index in *chosen (and the measured ms per step in
 * h_ms[0..max_out) if h_ms is not NULL).  The timed steps are ordinary steps of
 * the simulation: every variant evaluates a cell's update with the same
 * arithmetic (tiled shapes differ only in the order of the FP64 partial sums,
 * hence in the last bits of the mean density of Eq. 9; the two forms agree to
 * FP32 rounding).  Synchronises the stream. */
enum { HLB_KIND_SPLIT = 0, HLB_KIND_FUSED = 1, HLB_KIND_MARCH = 2 };
int hlb_tile_variants(int* h_tile_w, int* h_tile_h, int* h_threads, int max_out);
int hlb_variant_kind(int v);
int hlb_variant_energy_rows(int v);
hlb_status hlb_autotune(hlb_domain* d, int steps_per_variant, int* chosen, float* h_ms, int max_out);
hlb_status hlb_batch_autotune(hlb_batch* b, int steps_per_variant, int* chosen, float* h_ms, int max_out);

/* Select variant v (0 <= v < hlb_tile_variants(...)) for later steps without
 * timing anything, e.g. to reproduce a launch configuration under a profiler.
 * HLB_EINVAL for a NULL handle, v out of range, or a variant the handle cannot
 * use (a row-marching one on a lattice wider than 512 columns; a split or
 * row-marching one with the isotropic scheme; a fused one in a batch with
 * N > 1). */
hlb_status hlb_set_tile_variant(hlb_domain* d, int v);
hlb_status hlb_batch_set_tile_variant(hlb_batch* b, int v);

/* ------------------------------------------------------- no-allocation step
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory (a plug-in inside an application that owns
 * every allocation through its own pool, or a process whose device memory is
 * fully reserved up front).  One coupled step, as the fused tiled kernel of
 * hlb_step performs it, of a domain whose state lives in the caller's buffers:
 *   d_f_in / d_f_out   9 planes of nx*ny FP32 populations (plane q at offset
 *                      q*nx*ny), deviations f_q - w_q rho_v for
 *                      HLB_STORE_DEVIATION or the populations themselves for
 *                      HLB_STORE_PLAIN; solid rows are ignored;
 *   d_T_in / d_T_out   nx*ny FP32 temperature;
 *   d_ftop_in / _out   3*nx FP32 (populations 4, 7, 8 entering the top row at
 *                      the previous step, same storage form); needed only for
 *                      HLB_TOP_CONVECTIVE, else may be NULL;
 *   rho_ave, U         the lagged mean fluid density and outlet velocity
 *                      (h_out->rho_ave and max(0, h_out->u_top) of the previous
 *                      call);
 *   h_out              the step's FP64 diagnostics (synchronises the stream).
 * Sites (at most HLB_STATIC_MAX_SITES) give the wetting table as in
 * hlb_set_nucleation_sites.  All scratch (per-block FP64 partials, the device
 * diagnostics record, the wetting table) lives in one static device array of
 * HLB_STATIC_SCRATCH_BYTES inside the library, held by every GPU that loads it
 * until exit; no call allocates.  Limits: nx <= HLB_STATIC_MAX_NX and at most
 * 17,549 tiles of 52 x 28 cells (about 25.5 million cells); larger lattices
 * return HLB_EINVAL.  Every call resolves the array's address on the current
 * device (cudaGetSymbolAddress, which allocates nothing); the first call on a
 * device also sets that device's kernel attributes, so make it before any
 * stream capture.  Each call reads the diagnostics record back to h_out and
 * synchronises the stream before it returns.  Every call shares the array and
 * clears what must start at zero; calls that overlap on the GPU race. */
#define HLB_STATIC_SCRATCH_BYTES (1u << 20)
#define HLB_STATIC_MAX_NX 16384
#define HLB_STATIC_MAX_SITES 32
hlb_status hlb_step_static(const hlb_params* p, int n_sites, const hlb_site* h_sites, const float* d_f_in,
                           float* d_f_out, const float* d_T_in, float* d_T_out, const float* d_ftop_in,
                           float* d_ftop_out, double rho_ave, double U, hlb_diag_record* h_out, void* stream);

const char* hlb_strerror(hlb_status s);

#ifdef __cplusplus
}
#endif
#endif /* HLB_H */
