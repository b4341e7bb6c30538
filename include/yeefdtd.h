/*
 * yeefdtd.h -- C ABI of the B300 Yee FDTD transmission-line library.
 *
 * The library advances Maxwell's equations on a Yee grid (Yee 1966, cited in
 * Sec. II-A of Sawant et al., arXiv 2208.04371) with per-edge permittivity and
 * conductivity, PEC ground and conductors, absorbing CPML slabs, a soft port
 * source, and per-step port voltage / current integrals feeding running DFTs,
 * and extracts the power-mode S*, the 50-ohm S, Z_c and the phase delay from
 * them (Sec. II-A, Eq. 1-6, 8).
 *
 * Conventions (every call):
 *   - returns a yf_status; YF_OK == 0.  yf_last_error() gives a message for the
 *     last failing call on the calling thread.  Nothing aborts, nothing throws.
 *   - handles are opaque and owned by the library until their *_destroy call.
 *   - input arrays are caller-owned and copied (or fully consumed) during the call;
 *     output arrays are caller-allocated.  Where a yf_mem argument is present the
 *     pointer may be host (YF_HOST) or device (YF_DEVICE) memory.
 *   - all physical quantities are SI doubles.
 *   - grid frame: nx x ny x nz cells; E_x(i+1/2,j,k), E_y(i,j+1/2,k),
 *     E_z(i,j,k+1/2), H_x(i,j+1/2,k+1/2), H_y(i+1/2,j,k+1/2), H_z(i+1/2,j+1/2,k).
 *     Field arrays exchanged through the ABI use the compact shape
 *     (nz+1) x (ny+1) x (nx+1), x fastest; entries outside a component's own
 *     index range are zero.  Propagation of the ports is along x.
 *   - the stream passed at creation orders all device work of the handle; a NULL
 *     stream makes the library create and own a non-blocking stream.
 */
#ifndef YEEFDTD_H
#define YEEFDTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    YF_OK = 0,
    YF_E_INVALID = 1,      /* bad argument (sizes, indices, NULL pointers)            */
    YF_E_OOM = 2,          /* device or host allocation failed                         */
    YF_E_CUDA = 3,         /* a CUDA runtime call failed                               */
    YF_E_STATE = 4,        /* wrong call order (e.g. add_port after the first step)    */
    YF_E_TIMEOUT = 5,      /* a bounded device-side wait gave up                       */
    YF_E_UNSTABLE = 6,     /* Courant limit exceeded, or non-finite port samples       */
    YF_E_UNSUPPORTED = 7   /* valid request this build does not implement             */
} yf_status;

typedef enum { YF_FP32 = 0, YF_FP64 = 1 } yf_prec;
typedef enum { YF_HOST = 0, YF_DEVICE = 1 } yf_mem;
typedef enum { YF_BC_PEC = 0, YF_BC_PML = 1 } yf_bc;

/* field component ids for yf_read_fields / yf_write_fields */
enum { YF_EX = 0, YF_EY = 1, YF_EZ = 2, YF_HX = 3, YF_HY = 4, YF_HZ = 5 };

typedef enum {
    YF_WAVE_NONE = 0,
    YF_WAVE_DIFF_GAUSS = 1,   /* Eq. 3: s(t) = -2 (t-t0)/sigma exp(-(t-t0)^2/sigma^2); p0 = sigma      */
    YF_WAVE_GAUSS_SINE = 2,   /* s(t) = sin(2 pi f0 (t-t0)) exp(-((t-t0)/tau)^2), tau = 2/(pi bw);
                                 p0 = f0, p1 = bw                                                    */
    YF_WAVE_TABLE = 3         /* table[n] = s((n+1) dt); zero past the end                             */
} yf_wave_kind;

typedef struct {
    int kind;                 /* yf_wave_kind                                              */
    double amplitude;         /* A: E_z += A s(t) on every source edge                     */
    double p0, p1;            /* kind-specific parameters, see yf_wave_kind                */
    double t0;                /* peak time; < 0 selects 3 sigma (Eq. 3) or 3 tau           */
    const double *table;      /* host pointer, YF_WAVE_TABLE only                          */
    long table_len;
} yf_waveform;

/* Port on the plane x = plane (Sec. II-A, Eq. 4).
 *   V = -(dy dz / width) * sum_{k0<=k<k1} sum_{j0<=j<=j1} w_j E_z(plane, j, k+1/2),
 *       w_j = 1/2 at j0 and j1 (trapezoid across the strip), sampled at t_{n+1};
 *   I = direction * mean of the two H loops at x = plane -+ 1/2, each the
 *       right-handed (about +x) rectangle y in {j0-m+1/2, j1+m-1/2},
 *       z in {kb-m+1/2, kt+m-1/2} one cell (m = margin) outside the conductor
 *       [kb, kt] (kb == kt for a zero-thickness sheet), sampled at t_{n+1/2}.   */
typedef struct {
    int axis;                 /* propagation axis; only 0 (x) is supported                  */
    int plane;                /* x index of the V surface, 1 <= plane < nx                  */
    int direction;            /* +1 incident wave travels +x, -1 travels -x                 */
    int j0, j1;               /* strip edges (node indices), j0 < j1                        */
    int k0, k1;               /* V surface rows k0 <= k < k1                                */
    int kb, kt;               /* conductor bottom and top nodes                             */
    int margin;               /* loop distance from the conductor in cells (>= 1)           */
    double width;             /* strip width [m]; <= 0 selects (j1 - j0) dy                 */
} yf_port_desc;

/* DFT accumulator kinds (bit mask for yf_set_dft_mode, single value for reads) */
enum { YF_DFT_FP64 = 1, YF_DFT_KAHAN32 = 2, YF_DFT_FP32 = 4 };

/* one port's DFT spectra, FP64, each of length nfreq (host pointers) */
typedef struct {
    const double *V_re, *V_im, *I_re, *I_im;
} yf_port_dfts;

typedef struct yf_grid yf_grid;

/* Message for the last failing call on this thread ("" if none). */
const char *yf_last_error(void);

/* CFL step (Sec. II-B and III): dt = courant / (c0 sqrt(dx^-2 + dy^-2 + dz^-2)).
 * courant must lie in (0, 1]. */
yf_status yf_courant_dt(double dx, double dy, double dz, double courant, double *dt);

/* Create a grid of nx*ny*nz cells (each >= 3).  dt <= 0 selects the Courant-0.99 step;
 * dt above the 3-D Courant limit returns YF_E_UNSTABLE.  All fields start at zero, all
 * edges vacuum, all six faces PEC. */
yf_status yf_grid_create(int nx, int ny, int nz, double dx, double dy, double dz, double dt,
                         yf_prec prec, void *stream, yf_grid **out);
yf_status yf_grid_destroy(yf_grid *g);
yf_status yf_grid_dt(yf_grid *g, double *dt);

/* Materials from a per-cell index (nz*ny*nx bytes, x fastest) into tables of nmat <= 256
 * entries (Sec. II-B, III: dielectrics, lossy metals).  Each E edge takes the mean eps_r
 * and sigma of the four cells sharing it and becomes PEC if any of them is PEC; the
 * update is the time-centred conductor form Ca = (1-L)/(1+L), Cb = (dt/eps)/(1+L),
 * L = sigma dt / (2 eps).  More than 255 distinct non-PEC edge materials returns
 * YF_E_UNSUPPORTED, as does any mu_r != 1.  mu_r may be NULL.
 * ids with where == YF_HOST (pageable or pinned) are copied into a device staging buffer of
 * nz*ny*nx bytes and the classes derived on a second stream the grid keeps for this, beside
 * work still queued on the grid's stream (the zeroing of yf_reset); the call returns after the
 * copy and the derivation have finished, so the caller may reuse its array at once, and the
 * grid's later work is ordered after them.  Device ids are read on the grid's stream.  A grid that has already stepped
 * (a re-solve after yf_reset) keeps that buffer until yf_grid_destroy; otherwise it is freed
 * before the call returns.  A small device scratch of the derivation (about 82 KB) is kept
 * per grid. */
yf_status yf_set_materials(yf_grid *g, const uint8_t *ids, yf_mem where, int nmat,
                           const double *eps_r, const double *sigma, const double *mu_r,
                           const uint8_t *is_pec);

/* Zero-thickness PEC sheet (a strip, Sec. II-B) on the plane normal_axis = index over
 * the node rectangle [lo0, hi0] x [lo1, hi1] of the two other axes in increasing order:
 * the tangential E edges on the sheet are held at zero. */
yf_status yf_add_pec_sheet(yf_grid *g, int normal_axis, int index, int lo0, int hi0, int lo1,
                           int hi1);

/* Boundary of each face (-x,+x,-y,+y,-z,+z): YF_BC_PEC, or YF_BC_PML (absorbing slab of
 * yf_set_pml's thickness, PEC wall behind it; Sec. II-A). */
yf_status yf_set_boundaries(yf_grid *g, const int bc[6]);

/* CPML slabs (Berenger's PML in stretched-coordinate form): ncells thick, polynomial
 * grading order, sigma_max = sigma_scale * 0.8 (order+1) / (eta0 d), kappa grading to
 * kappa_max, CFS alpha falling linearly from alpha_max.  Defaults: 8, 3, 1, 1, 0. */
yf_status yf_set_pml(yf_grid *g, int ncells, int order, double sigma_scale, double kappa_max,
                     double alpha_max);

/* Soft source (Sec. II-A, Eq. 3): after each E update, E_z(plane, j, k+1/2) += A s(t_{n+1})
 * for j0 <= j <= j1, k0 <= k < k1, skipping PEC edges.  axis must be 0. */
yf_status yf_set_source(yf_grid *g, int axis, int plane, int j0, int j1, int k0, int k1,
                        const yf_waveform *w);

/* Add a port with its own frequency list (host array of nfreq > 0 values in Hz).
 * Must precede the first yf_step. */
yf_status yf_add_port(yf_grid *g, const yf_port_desc *d, int nfreq, const double *freqs_hz,
                      int *port_id);

/* Which DFT accumulators run (mask of YF_DFT_*; default YF_DFT_FP64).  Before the first step. */
yf_status yf_set_dft_mode(yf_grid *g, int mask);

/* Kernel variant of the time step (default 2):
 *   0  reference form: one H kernel and one E kernel, updating the fields in place;
 *   1  fused: H and E of a step in one pass (2.5-D z-march over 32 x tile_y node columns,
 *      kseg z-planes per block), reading one field buffer and writing the other, planes
 *      staged in shared memory by ordinary loads;
 *   2  as 1, with the planes staged by TMA (cp.async.bulk.tensor) three planes ahead of the
 *      computation; a bounded wait that expires makes yf_sync return YF_E_TIMEOUT;
 *   3  as 2, skewed by one plane (H on plane t and E on plane t-1 per iteration, one block
 *      barrier per plane, CPML auxiliaries fetched ahead of the arithmetic);
 *   4  FP32 only: two time steps per pass over the inner box (the nodes at least three cells
 *      from every absorbing slab, wall, source plane and port plane): one kernel advances it
 *      from step n to n+2 in a single read of step n, while variant 2's kernels advance the
 *      rest of the grid one step at a time, with the port epilogue after each step.  Uses a
 *      third field buffer (6 (nz+1)(ny+1) px words more, px = nx+1 rounded up to 32, allocated here or at the first step and
 *      freed when another variant is set).  An odd remaining step runs as variant 2.  The
 *      two-step blocks take 2 kseg z-planes each unless yf_set_box_shape says otherwise.
 * tile_y in {4, 8, 16}, 1 <= kseg <= 64.  All variants compute the same update; results agree to
 * rounding.  Drops captured graphs; may be called between steps.  YF_E_INVALID for variant 4
 * on an FP64 grid or on one with 6 (nz+1)(ny+1) px >= 2^31 (32-bit offsets in its kernel). */
yf_status yf_set_variant(yf_grid *g, int variant, int tile_y, int kseg);

/* Variant 4: the shape of the two-step kernel's blocks.  tile_y = 8 (0 selects it) or 16 nodes
 * of y per block (32 of x either way; 8: two blocks per SM, 16: one block per SM, which
 * recomputes fewer halo nodes); planes >= 1 z-planes per block, or 0 for the default 2 kseg.
 * A tuning choice only: every shape gives the same fields bit for bit (each block
 * recomputes its halo from step-n data).  Longer segments re-read fewer halo planes; the
 * count of blocks decides how they pack onto the SMs and how much of the frame's first step
 * runs beside them.  The inner box's y range is aligned to the larger of tile_y and the
 * frame's tile height.  Drops captured graphs; may be called between steps.  YF_E_INVALID for
 * another tile_y or planes < 0. */
yf_status yf_set_box_shape(yf_grid *g, int tile_y, int planes);

/* Variant 4's inner box as node ranges x0, x1, y0, y1, z0, z1 (inclusive; all -1 when the
 * grid has no box, which then steps one step at a time).  Finalises the geometry like a first
 * yf_step.  YF_E_STATE unless variant 4 is set. */
yf_status yf_tb_box(yf_grid *g, int box[6]);

/* Autotuner (before the first step): times the TMA-staged fused step (variant 2) for
 * tile_y in {4, 8, 16} x kseg in {8, 16, 32} over `reps` steps each with CUDA events, keeps
 * the fastest, resets fields, auxiliaries, spectra and the step count to zero, and caches the
 * choice in the JSON file cache_path (NULL: no cache) under a key of precision, size bucket
 * (cells rounded up to a power of two) and presence of absorbing slabs; a cached key skips
 * the timing.  The chosen tile_y and kseg are returned (either pointer may be NULL), and the
 * grid is left on variant 2 with them (set variant 4 again afterwards to use the two-step
 * path with the chosen tile). */
yf_status yf_autotune(yf_grid *g, const char *cache_path, int reps, int *tile_y, int *kseg);

/* Advance n time steps asynchronously on the handle's stream (Sec. II-A time loop:
 * H half step, E half step, source, port sampling, DFT accumulation).  Steps are
 * replayed from captured CUDA graphs in chunks. */
yf_status yf_step(yf_grid *g, long n);

/* Wait for the handle's stream; YF_E_UNSTABLE if a port sample became non-finite. */
yf_status yf_sync(yf_grid *g);
yf_status yf_steps_done(yf_grid *g, long *n);

/* Copy one component (YF_EX..YF_HZ) out of / into the grid in the compact
 * (nz+1)(ny+1)(nx+1) layout, in the grid's precision (float or double).  Synchronous. */
yf_status yf_read_fields(yf_grid *g, int comp, void *dst, yf_mem where);
yf_status yf_write_fields(yf_grid *g, int comp, const void *src, yf_mem where);

/* Field energy monitor: sum over edges of eps E^2 plus sum over faces of mu0 H^2, times
 * the cell volume, in FP64 (deterministic two-pass reduction).  Synchronous. */
yf_status yf_energy(yf_grid *g, double *w);

/* Running DFT of port `port` (Sec. II-A, F[.] of Eq. 1-2):
 * X(f) = sum_n x(t_n) exp(-j 2 pi f t_n) dt over V(t_{n+1}) and I(t_{n+1/2}); the phase
 * is an exact 64-bit integer count of half steps.  kind selects one accumulator
 * (YF_DFT_*).  Host outputs of nfreq doubles each; synchronous. */
yf_status yf_read_port_dft(yf_grid *g, int port, int kind, double *V_re, double *V_im,
                           double *I_re, double *I_im);

/* Network parameters on the GPU in FP64 (Sec. II-A), host arrays:
 *   inc[j]        : DFTs at the driven port j of the incident (uniformised-line) run
 *   tot[j*N + i]  : DFTs at port i of the total run driven at port j (V used)
 * outputs (any may be NULL), complex values interleaved (re, im):
 *   S_star [F][N][N]  Eq. 1 (S*_ij = V_tra,i / V_inc,j sqrt(Z_r,j / Z_r,i), S*_jj = V_ref/V_inc)
 *   S      [F][N][N]  Eq. 5-6 renormalised to z_ref ("*" read as the new reference)
 *   Zr     [N][F]     Eq. 2 Z_r = V_inc / I_inc
 *   Zc     [F]        sqrt(B/C) of the ABCD matrix of S* (N == 2 only)
 *   tau    [F][N][N]  Eq. 8, theta = -unwrap(arg S*_ij) in degrees, i != j; 0 on the diagonal
 * N <= 8. */
yf_status yf_sparams(int nports, int nfreq, const double *freqs, const yf_port_dfts *inc,
                     const yf_port_dfts *tot, double z_ref, double *S_star, double *S, double *Zr,
                     double *Zc, double *tau);

/* Same extraction as yf_sparams, for callers that cannot allocate GPU memory: code that
 * enqueues work while a stream is being captured in global mode (where cudaMalloc is not
 * allowed), or programs whose device memory is owned by their own pool or arena.  The paper
 * has no counterpart; it is an interface addition of this library.
 *   - allocates nothing: no cudaMalloc / cudaFree.  All pointers are DEVICE pointers owned by
 *     the caller; complex values are interleaved (re, im):
 *       freqs [F]; V_inc, I_inc [N][F]; V_tot [N][N][F] (driven j, port i);
 *       S [F][N][N] and Zr [N][F] required; S_star [F][N][N], Zc [F] (N == 2) and
 *       tau [F][N][N] optional (NULL skips them).
 *   - its scratch (the S* matrix the phase-delay pass reads) is one fixed array per GPU,
 *     held from library load until process exit: nfreq * nports^2 <= 32768 complex entries
 *     (512 KiB); larger requests return YF_E_INVALID before any work is queued.
 *   - asynchronous on `stream` (NULL = legacy default stream); the caller synchronises.
 *   - every call made while `stream` is not capturing looks up the scratch's device address
 *     (cudaGetSymbolAddress) in the current context and records it; a call made while
 *     `stream` is capturing uses the recorded address.  So the first call in each context
 *     (each device, and again after anything that destroys the context, such as
 *     cudaDeviceReset) must come before any stream capture; otherwise YF_E_STATE.
 *   - an error already pending in the CUDA runtime is returned (and cleared) before any work
 *     is queued; an error after that names the launch that failed.
 *   - every call shares the one scratch array and overwrites all of it that it uses: calls
 *     that may overlap on the GPU (different streams, concurrent host threads) race; order
 *     them on one stream or synchronise between them. */
yf_status yf_sparams_noalloc(int nports, int nfreq, const double *freqs, const double *V_inc,
                             const double *I_inc, const double *V_tot, double z_ref,
                             double *S_star, double *S, double *Zr, double *Zc, double *tau,
                             void *stream);

/* Telegrapher's model of a two-port (end of Sec. II-A): per-unit-length R [ohm/m], L [H/m],
 * G [S/m], C [F/m] and, when gamma is non-NULL, the propagation constant gamma [1/m]
 * (complex interleaved, [F]) of a line of physical length `length` [m].
 *   S_star [F][2][2] and Zr [2][F]: host arrays, complex interleaved (as yf_sparams returns).
 *   S* -> Z (pseudo-waves with the port references) -> ABCD; gamma l = +-acosh((A + D)/2)
 *   + 2 pi j k.  acosh folds beta l into [0, pi], so the branch is continued from the lowest
 *   frequency (which must have beta l < pi, as for Eq. 8) along beta l ~ f, and alpha's sign
 *   follows from beta > 0; Z_c = sqrt(B/C), Re >= 0; R + j w L = gamma Z_c,
 *   G + j w C = gamma / Z_c.  Frequencies must be positive and increasing.  A frequency where
 *   the conversion is singular (I - S* not invertible, e.g. a matched lossless line at
 *   beta l = m pi) gives NaN there only.
 * FP64 on the GPU; synchronous. */
yf_status yf_rlcg(int nfreq, const double *freqs, const double *S_star, const double *Zr,
                  double length, double *gamma, double *R, double *L, double *G, double *C);

/* Uniform-line shortcut for a two-port grid driven at port 0 (incident and total runs
 * coincide; S*_11 = S*_22 = 0, S*_12 = S*_21; port 1's Z_r from the same forward wave).
 * Uses the FP64 accumulators and port 0's frequency list. */
yf_status yf_read_sparams(yf_grid *g, double z_ref, double *S_star, double *S, double *Zr,
                          double *Zc, double *tau);

/* yf_read_sparams from a chosen accumulator set (YF_DFT_FP64, YF_DFT_KAHAN32 or YF_DFT_FP32;
 * YF_E_STATE if that set was not enabled by yf_set_dft_mode).  The extraction itself is FP64
 * whichever accumulators fed it: this is how the precision study (FP32 fields, three DFT
 * accumulator precisions, Sec. 2's running transform over a million steps) compares them. */
yf_status yf_read_sparams_acc(yf_grid *g, int kind, double z_ref, double *S_star, double *S,
                              double *Zr, double *Zc, double *tau);

/* Start a new solve on the same grid: zero fields, CPML auxiliaries, DFT accumulators,
 * step count and error bits, and reopen the geometry (yf_set_materials and
 * yf_add_pec_sheet accept new input; sheets added before are dropped).  Boundaries,
 * PML, source, ports and captured graphs are kept.  The call first waits for the grid's queued
 * work; the zeroing itself is queued on the grid's stream (later work there follows it; the
 * host does not wait for it). */
yf_status yf_reset(yf_grid *g);

/* Tracing: run n steps without graphs, bracketing every kernel launch with CUDA events
 * on the handle's stream, and return the mean duration in ms per launch of each kernel
 * of a step (names via yf_kernel_name).  *nkern receives the number of kernels (<= 8).
 * Variant 4 runs max(1, n/2) pairs of steps and reports four entries: the box kernel (timed
 * on its own stream, one launch per pair), the first frame step (all its work kinds; it runs
 * beside the box kernel, so both times include that sharing), the second frame step (after
 * the box kernel) and the epilogue (mean of the two per pair). */
yf_status yf_profile_steps(yf_grid *g, long n, double *ms_per_launch, int *nkern);
const char *yf_kernel_name(yf_grid *g, int idx);

/* Number of kernel launches one yf_step issues per time step with the current variant and
 * tiling (the stencil launches plus the epilogue), for launch accounting.  Finalises the
 * geometry like a first yf_step would. */
yf_status yf_launches_per_step(yf_grid *g, int *n);

/* Exact number of kernel launches a yf_step(g, nsteps) issues from the current state (variant
 * 4 launches per pair of steps; yf_launches_per_step then gives the mean rounded up).
 * Finalises the geometry like yf_launches_per_step.  YF_E_INVALID for nsteps < 0. */
yf_status yf_launches(yf_grid *g, long nsteps, long *n);

/* Failure-detection check, no counterpart in the paper: one device thread waits, with the
 * library's bounded-wait rule (a %globaltimer limit, never an unbounded spin), for a flag that
 * is set beforehand when preset_flag != 0 and never set otherwise.  Returns YF_OK when the
 * flag was seen and YF_E_TIMEOUT when the wait gave up after limit_seconds (0 < limit <= 10);
 * either way the CUDA context stays usable.  Synchronous on the legacy default stream. */
yf_status yf_bounded_wait_check(int preset_flag, double limit_seconds);

/* Binary checkpoint of fields, CPML auxiliaries, DFT accumulators and the step count;
 * load requires a grid created and configured identically. */
yf_status yf_checkpoint_save(yf_grid *g, const char *path);
yf_status yf_checkpoint_load(yf_grid *g, const char *path);

/* ---- batched solve of many independent lines (one shared time step) --------------------
 * Each instance is configured exactly as a single grid would be (the fields below map to
 * yf_set_materials, yf_add_pec_sheet, yf_set_boundaries, yf_set_pml, yf_set_source and
 * yf_add_port); all instances advance together: per step one launch over the CPML-free
 * interior work of every instance, one over the CPML frames, one port epilogue with a block
 * per instance; chunks of steps replay from captured CUDA graphs. */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    const uint8_t *ids;           /* host, nz*ny*nx; NULL keeps vacuum */
    int nmat;
    const double *eps_r, *sigma, *mu_r;   /* mu_r may be NULL */
    const uint8_t *is_pec;        /* may be NULL */
    int nsheets;
    const int *sheets;            /* nsheets x {normal_axis, index, lo0, hi0, lo1, hi1} */
    int bc[6];
    int pml_cells, pml_order;
    double pml_sigma_scale, pml_kappa_max, pml_alpha_max;
    int src_plane, src_j0, src_j1, src_k0, src_k1;
    yf_waveform src;              /* kind YF_WAVE_NONE: no source */
    int nports;
    const yf_port_desc *ports;
    int nfreq;                    /* one frequency list shared by the instance's ports */
    const double *freqs;
} yf_instance_desc;

typedef struct yf_batch yf_batch;

/* dt <= 0 selects 0.99 of the smallest Courant limit among the instances; a dt above any
 * instance's limit returns YF_E_UNSTABLE.  Fields of every instance start at zero. */
yf_status yf_batch_create(int n, const yf_instance_desc *d, double dt, yf_prec prec, void *stream,
                          yf_batch **out);
yf_status yf_batch_destroy(yf_batch *b);
/* Tile height (4, 8, 16) and z-planes per work item; defaults 8 and 16. */
yf_status yf_batch_set_tiling(yf_batch *b, int tile_y, int kseg);
/* Variant 4 for every instance (FP32 batches, before the first step; the default is the
 * one-step path): each instance keeps a third field buffer, and its inner box (the same box as
 * a single grid's variant 4, one z segment per tile column) advances two steps per pass while
 * its CPML frame and the other instances' small grids take one; the instances' results equal
 * their single-grid variant-4 results.  Returns YF_E_INVALID for other variants or FP64,
 * YF_E_STATE after a step. */
yf_status yf_batch_set_variant(yf_batch *b, int variant);
yf_status yf_batch_step(yf_batch *b, long n);
/* YF_E_TIMEOUT / YF_E_UNSTABLE as for single grids (any instance). */
yf_status yf_batch_sync(yf_batch *b);
yf_status yf_batch_info(yf_batch *b, int *n, long *cells, double *dt, long *steps);
/* The instance's grid handle (owned by the batch) for the single-grid read-out calls
 * (yf_read_fields, yf_read_port_dft, yf_read_sparams, yf_energy). */
yf_status yf_batch_grid(yf_batch *b, int inst, yf_grid **g);
yf_status yf_batch_read_port_dft(yf_batch *b, int inst, int port, int kind, double *V_re,
                                 double *V_im, double *I_re, double *I_im);
/* As yf_autotune, for the batch (key over the batch's total cells). */
yf_status yf_batch_autotune(yf_batch *b, const char *cache_path, int reps, int *tile_y, int *kseg);

#ifdef __cplusplus
}
#endif
#endif
