/*
 * hv.h - C ABI of libhv, a GB300 (sm_103a) implementation of the per-step ion
 * loop of the kinetic-ion / massless-fluid-electron hybrid particle-in-cell
 * method of Hybrid-VPIC (arXiv 2305.05600).
 *
 * One step n -> n+1 (Sec. 2.2 of the paper):
 *   [every sort_every steps: stable counting sort of the ions by supercell
 *    key (tile, then cell in the tile) of their predicted cells]
 *   gather E^n, B^n at x^n with the particle shape (NGP Eq. 13, QS Eqs. 17-19,
 *   or CIC on cell centres) -> non-relativistic Boris push (Eq. 9) ->
 *   deposit n, J_i at the half-step position (App. B) -> move (Eq. 10)
 *   -> linear extrapolation of the moments (Eq. 11) -> Faraday's law (Eq. 5)
 *   subcycled nsub times, E from Ohm's law (Eqs. 2-4, 6) with the density
 *   floor -> E^{n+1} = Ohm(B^{n+1}, n^{n+1}, J^{n+1}).
 *
 * Conventions for every entry point:
 *  - Units are normalised Alfvenic units (e = m_p = mu_0 = n_0 = 1, lengths in
 *    d_i, time in 1/Omega_ci, velocity in v_A, B in B_0).
 *  - Cells are cell-centred (Sec. 2.2); the linear cell index is
 *    c = i + nx*(j + ny*k), x fastest; all boundaries are periodic (Sec. 2.3).
 *    2D runs are x-z planes with ny = 1; any axis may have one cell.
 *  - A particle is a cell index plus relative coordinates in [-1, 1) per axis
 *    (Sec. 2.2), x = x_c + d * Delta / 2; along a single-cell axis the
 *    coordinate is ignored and reported as 0.
 *  - Grids exchanged with the caller are float32, component-major
 *    [ncomp][nz][ny][nx].  Particle arrays are float32 SoA, [3][n] for
 *    vectors.
 *  - Pointers are borrowed for the duration of the call only; the library
 *    copies what it keeps.  `on_device` = 1 means the pointer is CUDA device
 *    memory, 0 means host memory.
 *  - No exception or process exit crosses the ABI.  Every call returns an
 *    hv_status; on failure hv_last_error() returns a thread-local message.
 *  - Work is enqueued on the stream given to hv_init_grid.  Device-side
 *    errors (a particle moving more than one cell per step, a non-finite
 *    particle) are latched in a device error word and reported by the next
 *    synchronising call (hv_moments, hv_diag, hv_get_ions).
 *  - A context is not thread-safe; use one context per stream.
 */
#ifndef HV_H
#define HV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hv_ctx hv_ctx; /* opaque; owned by the library */

typedef enum {
  HV_OK = 0,
  HV_EINVAL = 1,   /* bad argument (checked on the host before any work) */
  HV_ENOMEM = 2,   /* device allocation failed */
  HV_ECUDA = 3,    /* a CUDA runtime call failed */
  HV_ECFL = 4,     /* a particle moved more than one cell in a step, or the
                      whistler limit Omega dt/nsub < dx^2/pi (Sec. 2.1) fails */
  HV_ENAN = 5,     /* a non-finite particle or diagnostic */
  HV_ETIMEOUT = 6, /* a bounded device wait gave up (error bit 8) */
  HV_ESTATE = 7    /* call out of order (e.g. loading ions after stepping) */
} hv_status;

typedef enum { HV_SHAPE_NGP = 0, HV_SHAPE_QS = 1, HV_SHAPE_CIC = 2 } hv_shape;

/* Simulation parameters (Secs. 2.1-2.2).  Layout is fixed (144 bytes). */
typedef struct {
  int32_t nx, ny, nz;   /* cells per axis, each >= 1, nx*ny*nz < 2^31 */
  int32_t nsub;         /* field subcycles per particle step (Sec. 2.1), >= 1 */
  double dx, dy, dz;    /* cell sizes in d_i (> 0); dy is used as given */
  double dt;            /* particle time step in 1/Omega_ci (> 0) */
  double Te;            /* electron temperature: p_e = Te * n^gamma_e (Eq. 6) */
  double gamma_e;       /* 1 isothermal, 5/3 adiabatic */
  double eta, eta_h;    /* resistivity and hyper-resistivity (Eq. 3) */
  double n_floor;       /* density floor n_f in Ohm's law (Sec. 2.1) */
  int32_t shape;        /* hv_shape */
  int32_t smooth_passes;/* binomial passes applied to deposited moments */
  int32_t sort_every;   /* sort ions by cell every this many steps; 0 never.
                           The cell an ion is sorted by is its cell moved by
                           at most one cell along each axis toward where it
                           is predicted to be 0.6875 sort intervals later:
                           along an axis of more than one cell, by +1 when
                           off + v * (float)(1.375 * sort_every * dt / Delta)
                           >= 1 and by -1 when it is < -1 (FP32, product and
                           sum rounded separately; the stored v, u with
                           relativistic particles), periodically.  Not with
                           open faces. */
  int32_t field_smooth_passes; /* binomial passes applied to copies of E^n and
                           B^n that the push gathers (the self-consistent
                           field smoothing of Sec. 2.2); the field state is
                           not smoothed; 0 off, at most 64 */
  uint64_t seed;        /* key of the random numbers of injection through
                           open faces (hv_set_injection) */
  int32_t pe_eq;        /* 1: the electron pressure is a field advanced with
                           the electron energy equation (Sec. 2.1, Eq. dpdt)
                           in the field subcycles; 0: p_e = Te n^gamma_e */
  int32_t ohm_model;    /* 0: hybrid Ohm's law (Eq. 2);
                           1: electrostatic E = -grad p_e / n_e (Sec. 4, Eq.
                              esohm, without collision terms), B not advanced
                              and kept at its loaded value;
                           2: resistive background E = eta (curl B - J_k)
                              (App. A), J_k the deposited current of the
                              kinetic species */
  double kappa;         /* heat conductivity of the electron energy
                           equation (>= 0) */
  int32_t relativistic; /* 1: the particles carry u = gamma v (loaded and
                           returned in place of v) and move with the
                           relativistic Boris push (App. A) */
  int32_t open_faces;   /* bit a set (a = 0 x, 1 y, 2 z): both faces of axis a
                           are open (Sec. 2.3) instead of periodic: one ghost
                           cell beyond each face copies B1, B0 and the
                           moments of its interior neighbour, Ohm's law there
                           drops the derivatives normal to the face, deposits
                           beyond the face fold onto the cell next to it, and
                           an ion that ends a step beyond it leaves the run;
                           ions enter through hv_set_injection.  Only with
                           ohm_model = 0, pe_eq = 0, no smoothing, no
                           relativistic push and more than one cell along the
                           axis (HV_EINVAL otherwise); 0: all periodic */
  double c_light;       /* speed of light in the velocity unit, > 0 when
                           relativistic (ignored otherwise) */
} hv_params;

/* FP64 diagnostics of the last completed step (or of the start-up state). */
typedef struct {
  int64_t step;      /* completed steps */
  double t;          /* step * dt */
  double W_K;        /* sum over ions of 1/2 m w |v^{n+1/2}|^2 (relativistic:
                        m w (gamma - 1) c^2) */
  double P[3];       /* sum over ions of m w v^{n+1/2} (relativistic: m w u) */
  double charge;     /* sum over cells of n^{n+1/2} V_c (= sum q w) */
  double W_B;        /* sum over cells of 1/2 |B^{n+1}|^2 V_c (total field) */
  double max_divB;   /* max over cells of |div_c B^{n+1}| (centred, Eq. 12;
                        of B1 when an external field is set) */
  int32_t err_word;  /* device error bits: 1 CFL, 2 non-finite particle,
                        4 corrupt cell index, 8 bounded wait gave up,
                        16 no free slot for injected ions */
  int32_t pad;
} hv_diag_t;

/* Accumulated device time per phase while profiling is on, and the number
 * of kernels launched.  Phases are timed with CUDA events on the context
 * stream; a sort issued ahead of its step on the library's side stream is
 * timed with events on that stream, so ms_sort is the sorts' own duration
 * even where they overlap the field phase (ms_field then includes the
 * overlap).  Injection through open faces counts with the moment post
 * (ms_moments, n_moments), so that ms_push / n_push is the push kernel's. */
typedef struct {
  double ms_sort, ms_push, ms_moments, ms_field, ms_ohm, ms_diag;
  int64_t n_sort, n_push, n_moments, n_field, n_ohm, n_diag; /* launches */
  int64_t steps;
  int64_t launches;  /* all library kernel launches since profiling began */
} hv_prof_t;

/* Layout facts of a context. */
typedef struct {
  int64_t ncell;      /* nx * ny * nz */
  int32_t tile[3];    /* supercell tile extents (x, y, z) of the ion order */
  int32_t ntiles;
  int32_t nspecies;
  int32_t pad;
  int64_t n[8];       /* ions per species (with open faces: particle slots,
                         live and free; hv_get_ions counts the live ions) */
  int64_t step;       /* completed steps */
} hv_info_t;

/* Device allocation hook used for every library-owned buffer.  alloc returns
 * NULL on failure.  `stream` is the context stream (cudaStream_t).  When no
 * hook is installed the library uses cudaMallocAsync / cudaFreeAsync. */
typedef void *(*hv_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*hv_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

/* Install (or, with NULLs, remove) the process-wide allocation hook.  Takes
 * effect for allocations made by later calls. */
hv_status hv_set_allocator(hv_alloc_fn alloc, hv_free_fn free_fn, void *user);

/* Create a context for the grid and physics in *p on the current CUDA device.
 * B0_host: initial magnetic field [3][nz][ny][nx] in host memory, or NULL for
 * the uniform field (1, 0, 0).  cuda_stream: a cudaStream_t (NULL = legacy
 * default stream).  Validates p (HV_EINVAL) and the whistler time-step limit
 * Omega_ci (dt/nsub) < min(dx,dy,dz)^2 / pi over axes with more than one cell
 * (Sec. 2.1; HV_ECFL) for the hybrid Ohm's law; with the electron energy
 * equation also h (gamma_e - 1) kappa / n_floor * sum 4/Delta^2 <= 2, and
 * for the resistive background h eta sum 4/Delta^2 <= 2 (explicit-midpoint
 * stability of the diffusion terms; HV_ECFL).  On success *out owns the
 * device state. */
hv_status hv_init_grid(const hv_params *p, const float *B0_host, void *cuda_stream,
                       hv_ctx **out);

/* Split the magnetic field as B = B0 + B1 (Sec. 2.3): B0_host [3][nz][ny][nx]
 * (host memory) is a fixed external field, for example the vacuum field of
 * coils or of a planet.  The field given to hv_init_grid stays the initial
 * total field; from this call on the library advances only B1 = B - B0 with
 * Faraday's law and takes the current in Ohm's law (Hall, resistive and
 * hyper-resistive terms) from J = curl B1, while the cross products of Ohm's
 * law and the push use the total field.  hv_moments reports the total
 * field; hv_diag reports W_B of the total field and max |div B1|.  Only
 * before the first step and once per context (HV_ESTATE otherwise);
 * HV_EINVAL for a non-finite value.  Synchronises. */
hv_status hv_set_external_field(hv_ctx *ctx, const float *B0_host);

/* Contexts with open faces (hv_params.open_faces): grow the particle slots
 * of species `species` to `capacity` (at least its loaded ions, below
 * 2^31 - 4) so that ions injected through open faces (hv_set_injection)
 * find free slots; a step that runs out of slots latches error bit 16
 * (HV_ENOMEM at the next synchronising call).  Slots of absorbed ions are
 * freed at each sort.  After hv_load_ions, before the first step
 * (HV_ESTATE otherwise); HV_EINVAL for a periodic context or a bad size. */
hv_status hv_reserve_ions(hv_ctx *ctx, int32_t species, int64_t capacity);

/* Inject ions of species `species` through open face `face` (0 -x, 1 +x,
 * 2 -y, 3 +y, 4 -z, 5 +z) every step, as the paper re-injects particles at
 * open boundaries (Sec. 2.3): the flux of a drifting Maxwellian with density
 * n, flow u[3] (velocity units) and temperature T (thermal speed
 * sqrt(T / m)), ions of weight w.  Per face cell and step the expected count
 * is N = Gamma A dt / w, Gamma = n [vt/sqrt(2 pi) exp(-U^2/2vt^2) +
 * U/2 (1 + erf(U/(sqrt2 vt)))] with U the inward flow and A the face cell
 * area, rounded stochastically; each ion's inward speed follows the
 * flux-weighted distribution and its tangential velocity the Maxwellian,
 * it enters at a uniform time within the step (uniform tangential
 * position), is appended after the push and deposits from the next step on.
 * The random numbers are Philox4x32-10 words keyed by hv_params.seed at
 * counters (step, face cell, ion, species and face), so runs repeat
 * exactly.  Before the first step, up to 6 faces per species; HV_EINVAL for
 * a face of a periodic axis or bad values. */
hv_status hv_set_injection(hv_ctx *ctx, int32_t species, int32_t face, double n,
                           const double *u, double T, double w);

/* Append ion species number `species` (must equal the number of species
 * already loaded; up to 8) with charge q and mass m (q_s = Z_s e, m_s; Sec.
 * 2.1) and n macro-particles: cell[n] int32 in [0, ncell), off3 [3][n]
 * relative coordinates in [-1, 1) (ignored along single-cell axes),
 * v3 [3][n] velocities v^{-1/2} (u = gamma v for a relativistic context),
 * w[n] weights (Sec. 2.2).  The arrays are
 * copied to the device (on_device != 0: they are device pointers) and every
 * value is checked there before the call returns (HV_EINVAL on a bad index,
 * offset or non-finite value; nothing of the species is kept then).  The
 * library reorders ions as it steps (a stable sort by supercell key, see
 * hv_get_tile_offsets) and copies weights bit for bit.  Only before the first step
 * (HV_ESTATE afterwards). */
hv_status hv_load_ions(hv_ctx *ctx, int32_t species, double q, double m, int64_t n,
                       const int32_t *cell, const float *off3, const float *v3,
                       const float *w, int on_device);

/* Enqueue nsteps full steps on the context stream and return without
 * waiting.  The first call also performs the start-up: moments of the
 * loaded ions at x^0 with v^{-1/2} become n^{-1/2}, J^{-1/2}, and
 * E^0 = Ohm(B^0, n^{-1/2}, J^{-1/2}).  Returns errors of argument checks and
 * launches only; device errors appear at the next synchronising call.
 * Besides the context stream the library uses its own side stream for a
 * sort issued ahead of its step and for clearing a deposit buffer; the
 * context stream waits for that work before anything reads its results,
 * and hv_destroy waits for it too. */
hv_status hv_step(hv_ctx *ctx, int32_t nsteps);

/* Copy the current grids out (any pointer may be NULL): n_out [nz][ny][nx]
 * and J_out [3][...] are the last deposited (smoothed) half-step moments
 * n^{n-1/2}, J^{n-1/2}; E_out, B_out [3][...] are E^n, B^n.  Synchronises
 * the stream and reports latched device errors. */
hv_status hv_moments(hv_ctx *ctx, float *n_out, float *J_out, float *E_out, float *B_out,
                     int on_device);

/* Copy the electron pressure field p_e^n [nz][ny][nx] out (Sec. 2.1, Eq.
 * dpdt), when the context was created with pe_eq = 1 (HV_EINVAL otherwise;
 * HV_EINVAL also for a NULL pe_out).  on_device: pe_out is device memory.
 * Synchronises the stream and reports latched device errors. */
hv_status hv_electron_pressure(hv_ctx *ctx, float *pe_out, int on_device);

/* FP64 diagnostics of the state after the last step (Secs. 2.1-2.2).
 * Synchronises; returns HV_ECFL / HV_ENAN when the error word or a
 * diagnostic says so (the struct is still filled). */
hv_status hv_diag(hv_ctx *ctx, hv_diag_t *out);

/* hv_diag without the wait.  hv_diag_async enqueues the diagnostics of the
 * state after the last step, with a copy of them and of the device error
 * word to page-locked host memory that the context owns, and returns at
 * once; up to 4 may be pending (HV_ESTATE when 4 are).  hv_diag_wait waits
 * for the oldest pending one and fills *out as hv_diag does (out->step is
 * the step it describes), with hv_diag's return codes; HV_ESTATE when none
 * is pending.  A caller that enqueues step k + 1 before it waits for the
 * diagnostics of step k reads every step's result while the GPU keeps
 * working. */
hv_status hv_diag_async(hv_ctx *ctx);
hv_status hv_diag_wait(hv_ctx *ctx, hv_diag_t *out);

/* Copy species `species` out in the library's current particle order (the
 * order changes when ions are sorted; see hv_query): cell [n], off3 [3][n], v3 [3][n]
 * (v^{n-1/2}), w [n].  Any pointer may be NULL.  n_out (may be NULL)
 * receives the particle count.  Synchronises. */
hv_status hv_get_ions(hv_ctx *ctx, int32_t species, int64_t *n_out, int32_t *cell,
                      float *off3, float *v3, float *w, int on_device);

/* Learned moment filter (not in the paper; an addition to its binomial
 * smoothing of noisy moments, Sec. 2.2): a residual 3x3 convolutional
 * network 4 -> 16 -> 16 -> 4 with ReLU between layers and periodic padding,
 * applied to the deposited half-step moments m = (n, Jx, Jy, Jz) of the x-z
 * layout in place of the binomial passes:
 *   x = m / scale4,  h1 = bf16(relu(conv(bf16(x), W1) + b1)),
 *   h2 = bf16(relu(conv(h1, W2) + b2)),  f = conv(h2, W3) + b3,
 *   m' = m + scale4 * f,
 * except where n < gate_nmin or |scale4[0] f_n| > gate_rmax max(n, n_floor);
 * there m' is one (1/4, 1/2, 1/4) pass per axis of m.  conv is the periodic
 * cross-correlation out[o](i,k) = b[o] + sum_c sum_{a,b} W[o][c][b+1][a+1]
 * in[c](i+a, k+b).  params (host, 3492 floats, used as bf16):
 * W1[16][4][3][3] b1[16] W2[16][16][3][3] b2[16] W3[4][16][3][3] b3[4].
 * params = NULL turns the filter off.  HV_EINVAL for a 3D grid or bad
 * values.  Takes effect from the next deposit. */
hv_status hv_set_filter(hv_ctx *ctx, const float *params, const float *scale4, double gate_nmin,
                        double gate_rmax);

/* Apply the context's learned filter (with its gate) to moments m4
 * [4][nz][ny][nx] (n, Jx, Jy, Jz), writing y4 of the same shape; both in host
 * (on_device = 0) or device memory.  For inspection and training data.
 * HV_ESTATE when no filter is set.  Synchronises. */
hv_status hv_filter_moments(hv_ctx *ctx, const float *m4, float *y4, int on_device);

/* Training of the learned filter on pairs the method generates (a
 * low-particle-count deposit m and a high-count deposit t of the same state):
 * loss = mean over cells, channels and pairs of (m/s + f(m/s) - t/s)^2 with
 * the network of hv_set_filter (no gate).  The forward pass and the
 * backward-data convolutions run on bf16 tensor cores with FP32
 * accumulation; weight gradients are accumulated in FP32; Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8) updates FP32 master parameters and
 * refreshes the context's bf16 inference weights.
 * hv_filter_train_init: set the starting parameters (3492 floats, host) and
 * scales, reset Adam, and install the filter with its gate open.
 * hv_filter_grad: loss and gradient (3492 floats, host) at the current
 * parameters, without an update.  hv_filter_train_step: one Adam step with
 * learning rate lr.  m and t are [nb][4][nz][ny][nx] float32 (host or device
 * per on_device).  hv_filter_get_params: the FP32 master parameters.
 * The x-z layout only.  All synchronise. */
hv_status hv_filter_train_init(hv_ctx *ctx, const float *params, const float *scale4);
hv_status hv_filter_grad(hv_ctx *ctx, const float *m, const float *t, int32_t nb,
                         float *grad_out, double *loss_out, int on_device);
hv_status hv_filter_train_step(hv_ctx *ctx, const float *m, const float *t, int32_t nb,
                               double lr, double *loss_out, int on_device);
hv_status hv_filter_get_params(hv_ctx *ctx, float *params_out);

/* Fill *out with the context's layout: the library keeps ions sorted
 * tile-major (supercell tile index, then the linear cell inside the tile,
 * both x fastest, of each ion's predicted cell, see sort_every) whenever it
 * sorts them, with tile extents as reported. */
hv_status hv_query(const hv_ctx *ctx, hv_info_t *out);

/* The ion range of every supercell tile of species `species` in the
 * library's current particle order: tile_off [ntiles + 1] (host memory)
 * receives the first ion of each tile and, last, the ion count.  After a
 * sort these are the offsets of a stable counting sort of the ions'
 * supercell keys (the key of an ion is that of its predicted cell, see
 * sort_every; the key of a cell is its tile index times the cells per tile
 * plus its cell inside the tile, x fastest; hv_query gives the tile
 * extents); before the first sort they split the ions evenly.  The sort is
 * an ordering device of the GPU layout (the paper prescribes none; it
 * changes results only through FP32 summation order).  Synchronises and
 * reports latched device errors. */
hv_status hv_get_tile_offsets(hv_ctx *ctx, int32_t species, int32_t *tile_off);

/* Fault injection for testing the failure path: OR `bits` (a non-empty
 * combination of the hv_diag_t err_word bits 1, 2, 4, 8, 16) into the context's
 * device error word, as a kernel that detected the fault would.  The next
 * synchronising call reports it (hv_error_status gives the mapping).
 * HV_EINVAL for other bits.  Nothing on the GPU faults or waits. */
hv_status hv_inject_error(hv_ctx *ctx, int32_t bits);

/* The status that a synchronising call returns for device error word
 * `err_word` (hv_last_error() then names the cause), without a context or a
 * GPU: bit 2 non-finite -> HV_ENAN, else bit 1 -> HV_ECFL, else bit 4 ->
 * HV_ECUDA, else bit 8 -> HV_ETIMEOUT, else bit 16 -> HV_ENOMEM, else HV_OK. */
hv_status hv_error_status(int32_t err_word);

/* Turn per-phase CUDA-event timing on (1) or off (0); turning it on resets
 * the counters.  hv_profile_read synchronises and returns the totals. */
hv_status hv_profile(hv_ctx *ctx, int enable);
hv_status hv_profile_read(hv_ctx *ctx, hv_prof_t *out);

/* Release every device buffer of the context (NULL is allowed). */
void hv_destroy(hv_ctx *ctx);

/* Stable sort by key: the radix passes of the step's general sort path
 * (which sorts ions by supercell key the same way), on caller keys.  Not in
 * the paper; it is a device of the GPU layout.
 * keys [n] int32 in [0, nkeys) on the device; perm [n] receives the gather
 * permutation (keys[perm[i]] non-decreasing, equal keys in input order);
 * counts [nkeys] (may be NULL) receives the number of each key.  All three
 * pointers are device memory.  Scratch is allocated through the allocation
 * hook and released before return.  Runs on cuda_stream and synchronises it.
 * HV_EINVAL for n < 0, nkeys < 1 or a key out of range (checked on device,
 * perm is then unspecified). */
hv_status hv_sort_keys(const int32_t *keys, int64_t n, int32_t nkeys, int32_t *perm,
                       int32_t *counts, void *cuda_stream);

/* The same stable key sort as hv_sort_keys, for callers that cannot allocate
 * device memory: for example an application that hands the whole GPU to its
 * own memory pool up front, or a latency-critical loop that must not enter
 * the CUDA allocator because an allocation can synchronise the device.  This
 * entry point allocates nothing (no cudaMalloc, no allocation hook): its
 * scratch is one static device array of about 16.3 MB that every GPU which
 * loads the library holds until the process exits.  The paper has no
 * counterpart; it is an interface convenience.
 *   keys [n], perm [n], counts [nkeys] (may be NULL): device memory owned by
 *   the caller, as for hv_sort_keys; n <= 1,048,576, larger n is rejected
 *   with HV_EINVAL before any GPU work.
 * The first call on a device looks up the array's device address (one
 * cudaGetSymbolAddress per device); make that first call before any stream
 * capture.  All calls share the one array and it keeps the last call's
 * contents (the call clears what must start at zero), so calls that overlap
 * on the GPU, from two streams or two threads, race and must be serialised
 * by the caller.  Runs on cuda_stream and synchronises it. */
hv_status hv_sort_keys_noalloc(const int32_t *keys, int64_t n, int32_t nkeys, int32_t *perm,
                               int32_t *counts, void *cuda_stream);

/* Thread-local description of the last failure (never NULL). */
const char *hv_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HV_H */
