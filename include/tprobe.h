/*
 * tprobe.h -- C ABI of the GB300 (sm_103a) probed FWI-gradient library.
 *
 * Implements the low-memory adjoint-state gradient of Louboutin & Herrmann,
 * "Ultra-low memory seismic inversion with randomized trace estimation"
 * (arXiv 2104.00794): constant-density acoustic finite differences, 2nd order
 * in time and 4th/8th order in space, whose forward and adjoint time loops
 * accumulate the wavefields projected onto r random time probes (Algorithm 1)
 * instead of storing the N x nt forward history (Eq. 3).
 *
 * Discrete system (shared reading of the paper, which gives no
 * discretisation): nodes nz x ny x nx (ny = 1 in 2-D), spacing h, zero
 * (Dirichlet) values outside the grid, flat index (z*ny + y)*nx + x.
 * Levels t = 0..nt-1 with u[0] = u[1] = 0 and, for t = 1..nt-2,
 *     u[t+1] = 2u[t] - u[t-1] + dt^2 v^2 (L u[t] + S^T q[t])
 * (Algorithm 1 line 1, operator f; L = centred Laplacian, Fornberg weights);
 * data d[t] = R u[t] (Eq. 2).  The adjoint (Algorithm 1 line 5, f^T) is the
 * exact transpose: lambda[nt] = lambda[nt+1] = 0 and, for j = nt-1..2,
 *     lambda[j] = 2 lambda[j+1] - lambda[j+2] + dt^2 v^2 (L lambda[j+1] + R^T s[j]).
 * With an absorbing layer (tp_grid.sponge > 0) both steps carry the damping
 * described at that field; the adjoint stays the exact transpose.
 * m = 1/v^2 is the squared slowness; every gradient returned is dJ/dm of
 * J = 1/2 sum_t ||R u[t] - d_obs[t]||^2 (Eq. 2), i.e. the negative of the
 * update direction delta m that Eq. 3 prints without a sign.
 *
 * Conventions for every entry point:
 *   - All array arguments are DEVICE pointers owned by the caller, unless a
 *     parameter says "host".  Nothing is allocated on the hot path: scratch
 *     space is the caller's workspace, sized by tp_workspace_bytes(); the one
 *     exception is tp_misfit_noalloc, whose scratch is a fixed 32 KiB array
 *     inside the library that all of its calls share.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t, NULL for
 *     the legacy default stream); results are ready once the stream is.
 *   - float = IEEE fp32; the wavefields are fp32 and the misfit / gradient
 *     norm are fp64 reductions.
 *   - Errors are returned as tp_status, never thrown; tp_last_error() gives a
 *     thread-local message for the last failing call on the calling thread.
 *   - Calls that share a workspace must not overlap on the device.
 */
#ifndef TPROBE_H
#define TPROBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TP_OK = 0,
  TP_ERR_ARG = 1,       /* invalid argument (sizes, pointers, geometry) */
  TP_ERR_UNSTABLE = 2,  /* CFL condition of the leapfrog scheme violated */
  TP_ERR_NOMEM = 3,     /* workspace smaller than tp_workspace_bytes() */
  TP_ERR_CUDA = 4,      /* a CUDA runtime call or kernel launch failed */
  TP_ERR_TIMEOUT = 5    /* a bounded device-side wait gave up */
} tp_status;

typedef enum {
  TP_PROBE_RADEMACHER = 0, /* +-1 entries (Eq. 1, random sign probes) */
  TP_PROBE_GAUSSIAN = 1,   /* Irwin-Hall(12) approximately normal entries */
  TP_PROBE_IDENTITY = 2,   /* Z = I, r = nt: reproduces Eq. 3 exactly */
  TP_PROBE_USER = 3        /* caller-supplied Z (e.g. QR range-finder probes) */
} tp_probe_kind;

typedef enum {
  TP_OP_FORWARD = 0,
  TP_OP_ADJOINT = 1,
  TP_OP_GRADIENT_PROBED = 2,
  TP_OP_GRADIENT_FULL = 3,
  TP_OP_PROBED_FORWARD = 4,   /* tp_probed_forward's transient workspace */
  TP_OP_PROBED_BACKWARD = 5   /* tp_probed_backward's transient workspace */
} tp_op;

/* Storage of the probe accumulators (ubar, vbar); the accumulation itself is
 * always fp32 (the tensor-core tile is added in fp32 before it is stored). */
typedef enum {
  TP_ACC_F32 = 0,         /* fp32: 4 B per value */
  TP_ACC_BF16 = 1,        /* bf16, round to nearest: 2 B per value */
  TP_ACC_BF16_KAHAN = 2,  /* bf16 value + bf16 compensation (the rounding error of
                             the stored value, carried to the next window): 4 B */
  TP_ACC_F32_FOLD = 3     /* one accumulator set (N r values instead of 2 N r, the
                             single-accumulator form of Algorithm 1 line 8): the
                             forward accumulators are fp32; before the adjoint
                             they are turned into ubar_i in place, and each adjoint
                             window's Q_w^T lambda is folded straight into the
                             gradient, g += sum_i ubar_i (Q_w^T lambda)_i, so vbar
                             is never stored.  Needs r <= 32.  tp_probed_backward
                             then overwrites the state's accumulators (the state
                             serves one backward call). */
} tp_acc;

/* Grid and time axis.  Eq. 2 (F(m; q) on this grid). */
typedef struct {
  int ndim;    /* 2 or 3 */
  int nx, ny, nz; /* nodes; ny must be 1 when ndim == 2 */
  float h;     /* grid spacing [m] */
  float dt;    /* time step [s] */
  int nt;      /* number of time levels (>= 3) */
  int order;   /* spatial order: 4 or 8 */
  float vmax;  /* > 0: caller-asserted max velocity used for the CFL check
                  (no device synchronisation); 0: the library reduces the
                  velocity on the device and synchronises the stream once */
  int form;    /* fp32 time stepping of the same scheme: TP_FORM_LEVELS keeps
                  (u[t], u[t-1]); TP_FORM_INCREMENT keeps (u[t], u[t] - u[t-1]),
                  so that the rounding of u is integrated once instead of
                  twice (more accurate over thousands of steps, one more
                  4-byte write per point and step); TP_FORM_COMPENSATED steps
                  the forward wavefield as a double-float u + e (fp32 level,
                  bf16 low part) with error-free sums, so that the rounding of
                  the stored levels is carried instead of lost (the probed
                  gradient applies the Laplacian to the probed forward field,
                  which amplifies that rounding); the adjoint keeps the levels
                  form.  TP_FORM_COMPENSATED needs a 2-D grid without an
                  absorbing layer whose shot fits one thread-block cluster
                  (tp_form_supported) */
  int sponge;  /* absorbing layer (not in the paper): width in cells on every
                  face but the top z = 0, which stays the zero-pressure free
                  surface; 0: none (the undamped scheme, bit for bit).  The
                  damping m * eta * du/dt, eta = sponge_eta ((w - d)/w)^2 at
                  distance d < w cells from a damped face, makes the step
                  (1+a) u[t+1] = 2u[t] - (1-a) u[t-1] + dt^2 v^2 (L u[t] + S^T q[t]),
                  a = eta dt / 2; the adjoint keeps the same form, and every
                  gradient is dJ/dm of the damped system */
  float sponge_eta; /* peak damping eta_max [1/s], >= 0 */
} tp_grid;

typedef enum { TP_FORM_LEVELS = 0, TP_FORM_INCREMENT = 1, TP_FORM_COMPENSATED = 2 } tp_form;

/* Acquisition of a batch of independent shots sharing one model.  S^T and R
 * of Eq. 2 / Algorithm 1: on-grid point sources and receivers. */
typedef struct {
  int nshots;          /* shots in the batch (>= 1) */
  int nsrc;            /* sources per shot (>= 1) */
  const int64_t* src;  /* device [nshots][nsrc] flat node indices */
  int nrec;            /* receivers per shot (>= 1) */
  const int64_t* rec;  /* device [nshots][nrec] flat node indices */
} tp_geom;

/* Probing matrix Q in R^{nt x r} of Eq. 4 / Algorithm 1, drawn per shot. */
typedef struct {
  int kind;            /* tp_probe_kind */
  int r;               /* probing vectors, 1..256 (== nt for IDENTITY) */
  int T;               /* time window of the probe GEMM: 32, 64 or 128 levels
                          (128 needs r <= 32); the ring holds T + 2 levels */
  uint64_t seed;       /* SplitMix64 seed (random kinds) */
  const float* Z_user; /* device [nshots][nt][r] when kind == TP_PROBE_USER */
  float scale;         /* estimator scale; 0 selects the default: 1/r for
                          random probes (Eq. 1), 1 for IDENTITY and USER */
  int acc;             /* tp_acc storage of the accumulators; all but F32 need r <= 32 */
} tp_probe;

/* TP_OK if this library can run `grid` (its form in particular) for batches
 * shaped like `geom` (only the counts of geom are read), else TP_ERR_ARG with
 * the reason in tp_last_error().  No device work. */
tp_status tp_form_supported(const tp_grid* grid, const tp_geom* geom);

/* Bytes of device workspace that `op` needs (0 on invalid arguments; see
 * tp_last_error).  `probe` is read only for the probed ops.  The workspace
 * must be 256-byte aligned. */
size_t tp_workspace_bytes(int op, const tp_grid* grid, const tp_geom* geom, const tp_probe* probe);

/* Forward modelling d = F(m; q) (Eq. 2; Algorithm 1 lines 0-3 without the
 * probe accumulation).  vel: [nz][ny][nx] m/s.  wavelet: [nshots][nt][nsrc]
 * source time functions q.  d_out: [nshots][nt][nrec], d_out[s][t] = R u[t]
 * (levels 0 and 1 are zero). */
tp_status tp_forward(const tp_grid* grid, const tp_geom* geom, const float* vel,
                     const float* wavelet, float* d_out, void* ws, size_t ws_bytes, void* stream);

/* Adjoint q = F^T s (Algorithm 1 lines 4-7 without the probe accumulation).
 * d_in: [nshots][nt][nrec] adjoint sources s.  q_out: [nshots][nt][nsrc],
 * q_out[s][t] = S lambda[t+1] for t = 1..nt-2 and 0 for t = 0, nt-1, so that
 * <F q, s> = <q, F^T s> holds to rounding. */
tp_status tp_adjoint(const tp_grid* grid, const tp_geom* geom, const float* vel,
                     const float* d_in, float* q_out, void* ws, size_t ws_bytes, void* stream);

/* Probed gradient (Algorithm 1, Eq. 4) summed over the batch's shots:
 *   grad[x] = - scale * sum_s sum_i ubar_s[x,i] vbar_s[x,i],
 *   ubar_s[x,i] = sum_{k=2}^{nt-1} Q_s[k,i] udd_s[k,x],  vbar likewise with lambda_s,
 * where udd[k] = (u[k] - 2u[k-1] + u[k-2]) / dt^2 and lambda is driven by the
 * residual d - d_obs.  grad: [nz][ny][nx] (dJ/dm).  misfit, gnorm: optional
 * DEVICE doubles receiving J = 1/2 ||d - d_obs||^2 and ||grad||_2.
 * d_obs: [nshots][nt][nrec].  Memory: 2 N r probe accumulators per shot plus
 * a (T + 2)-level ring, instead of the N nt history of tp_gradient_full. */
tp_status tp_gradient_probed(const tp_grid* grid, const tp_geom* geom, const tp_probe* probe,
                             const float* vel, const float* wavelet, const float* d_obs,
                             float* grad, double* misfit, double* gnorm, void* ws,
                             size_t ws_bytes, void* stream);

/* Conventional adjoint-state gradient (Eq. 3) with the full N x nt forward
 * history kept in the workspace; same arguments and outputs as
 * tp_gradient_probed without the probes. */
tp_status tp_gradient_full(const tp_grid* grid, const tp_geom* geom, const float* vel,
                           const float* wavelet, const float* d_obs, float* grad, double* misfit,
                           double* gnorm, void* ws, size_t ws_bytes, void* stream);

/* Algorithm 1 split at the residual, for callers that drive the adjoint
 * source themselves (e.g. a torch.autograd.Function whose backward receives
 * dL/dd).  `state` is a caller-owned device buffer of tp_probed_state_bytes()
 * (256-byte aligned) holding what must survive between the two halves: the
 * probes Q and the forward accumulators ubar (2 N r values with vbar, Section
 * "Memory estimates"); nothing else is kept.
 *
 * tp_probed_forward: lines 0-3.  d_out [nshots][nt][nrec] = F(m; q) and ubar
 * into `state`.  ws: tp_workspace_bytes(TP_OP_PROBED_FORWARD, ...).
 * tp_probed_backward: lines 4-8 with adjoint source adj_src [nshots][nt][nrec]
 * (for J = 1/2 |d - d_obs|^2 that is the residual).  grad [nz][ny][nx]
 * receives dJ/dm (wrt_velocity = 0) or dJ/dv = dJ/dm * (-2 / v^3)
 * (wrt_velocity = 1); gnorm (optional, device) its fp64 norm.
 * ws: tp_workspace_bytes(TP_OP_PROBED_BACKWARD, ...).  The same grid, geom,
 * probe and vel must be passed to both halves. */
size_t tp_probed_state_bytes(const tp_grid* grid, const tp_geom* geom, const tp_probe* probe);
tp_status tp_probed_forward(const tp_grid* grid, const tp_geom* geom, const tp_probe* probe,
                            const float* vel, const float* wavelet, float* d_out, void* state,
                            size_t state_bytes, void* ws, size_t ws_bytes, void* stream);
tp_status tp_probed_backward(const tp_grid* grid, const tp_geom* geom, const tp_probe* probe,
                             const float* vel, const float* wavelet, const float* adj_src,
                             int wrt_velocity, float* grad, double* gnorm, void* state,
                             size_t state_bytes, void* ws, size_t ws_bytes, void* stream);

/* The data residual and misfit between the halves (Eq. 2): d becomes the
 * residual d - d_obs in place, and J = 1/2 sum_i (d[i] - d_obs[i])^2 is
 * reduced in fp64 in a fixed order and written to the DEVICE double *misfit.
 * With d = the d_out of tp_probed_forward, the residual is the adj_src of
 * tp_probed_backward, and the three calls give bit for bit what
 * tp_gradient_probed gives (same kernels, same order): a caller can then
 * upload d_obs while the forward half runs.  d, d_obs: device float arrays
 * of n samples (any layout, e.g. [nshots][nt][nrec]); ws: caller-owned device
 * workspace of tp_residual_workspace_bytes() bytes, 256-byte aligned (fp64
 * partial sums).  Errors: TP_ERR_ARG (NULL pointer, n < 1, misaligned ws),
 * TP_ERR_NOMEM (ws too small), TP_ERR_CUDA (launch failed). */
size_t tp_residual_workspace_bytes(void);
tp_status tp_residual(float* d, const float* d_obs, int64_t n, double* misfit, void* ws, size_t ws_bytes,
                      void* stream);

/* Imaging conditions on the probed wavefields (§Imaging conditions, Eq. 5:
 * a linear operator D that acts on space only commutes with probing,
 * Q^T (D u) = D (Q^T u)).  tp_probed_image applies D to the r probed fields
 * P_i = sum_{j=2}^{nt-2} Q[j+1, i] u[j] (the state of tp_probed_forward) and
 * V_i = sum_{k=2}^{nt-1} Q[k, i] lambda[k] (an adjoint run driven by adj_src,
 * [nshots][nt][nrec]) instead of to nt snapshots:
 *   image(x) = scale * sum_shots sum_i <D P_i(x), D V_i(x)>,
 * an estimate of sum_shots sum_j <D u[j](x), D lambda[j+1](x)> (exact for
 * TP_PROBE_IDENTITY).  image: device [nz][ny][nx] fp32.  The probe must use
 * TP_ACC_F32 storage; ws: tp_workspace_bytes(TP_OP_PROBED_BACKWARD, ...);
 * the same grid, geom, probe and vel as the forward half.  The state is only
 * read.  Errors as tp_probed_backward, TP_ERR_ARG for an unknown cond. */
typedef enum {
  TP_IMAGE_CORRELATION = 0,  /* D = identity: cross-correlation image */
  TP_IMAGE_GRADIENT = 1      /* D = spatial gradient (centred first differences of the
                                grid's order, divided by h), summed over the axes */
} tp_image_cond;
tp_status tp_probed_image(const tp_grid* grid, const tp_geom* geom, const tp_probe* probe, const float* vel,
                          const float* adj_src, int cond, float* image, const void* state, size_t state_bytes,
                          void* ws, size_t ws_bytes, void* stream);

/* Range-finding probes of Eq. 6 for every shot: Q_s = qr(D_s D_s^T Z_s), where
 * D_s = d_obs[s] is the observed record as an nt x nrec matrix (time x
 * receivers) and Z_s the random probes that `probe` (kind RADEMACHER or
 * GAUSSIAN, r <= 32, seed) draws for shot s.  Q: device [nshots][nt][r] fp32
 * with orthonormal columns and diag(R) > 0 (computed in fp64: two reductions
 * for D (D^T Z), then Gram-Schmidt applied twice).  Pass Q back as
 * TP_PROBE_USER probes (scale 1).  ws: tp_qr_workspace_bytes(); a numerically
 * rank-deficient record leaves zero columns and sets a flag that
 * tp_workspace_status reports as TP_ERR_ARG. */
size_t tp_qr_workspace_bytes(int nt, int nrec, int nshots, int r);
tp_status tp_qr_probes(const tp_probe* probe, int nt, int nrec, int nshots, const float* d_obs, float* Q,
                       void* ws, size_t ws_bytes, void* stream);

/* The probing matrix that tp_gradient_probed draws for shot `shot`
 * (Eq. 1 probes from SplitMix64; Z[t][i], [nt][r], unscaled).  For
 * TP_PROBE_USER it copies the caller's Z. */
tp_status tp_probes(const tp_probe* probe, int nt, int shot, float* Z, void* stream);

/* Data misfit J = 1/2 sum_i (d_syn[i] - d_obs[i])^2 over n samples, written
 * to the DEVICE double *misfit, computed without any workspace.  The paper has
 * no counterpart: this entry point exists for callers that cannot allocate
 * device memory where they need the misfit -- code that gets all of its device
 * memory from a host framework's own pool and may not allocate by itself, or a
 * latency-critical loop where an allocation (and the synchronisation it can
 * bring) is not acceptable.  Its scratch (one fp64 partial per 65536 samples)
 * is a fixed 32 KiB array inside the library, held on every GPU that loads the
 * library until the process exits; so n may be at most 268,435,456 samples
 * (TP_ERR_ARG beyond).  Each call made outside stream capture looks the
 * array up on the current device (cudaGetSymbolAddress), so a device reset
 * between calls is harmless; a call made during capture uses the address of
 * the last call outside capture on that device, so make the first call on a
 * device before any capture, and none across a device reset during capture.
 * Calls share the array: calls that overlap on the GPU race and must
 * be ordered by the caller.  d_syn, d_obs: device float arrays of n samples
 * (any layout, e.g. [nshots][nt][nrec]).  Errors: TP_ERR_ARG (NULL pointer,
 * n < 1 or too large), TP_ERR_CUDA (lookup or launch failed). */
tp_status tp_misfit_noalloc(const float* d_syn, const float* d_obs, int64_t n, double* misfit, void* stream);

/* Synchronises `stream` and reports whether a bounded device-side wait in
 * the last call on this workspace gave up (TP_ERR_TIMEOUT) or not (TP_OK);
 * clears the flag. */
tp_status tp_workspace_status(void* ws, size_t ws_bytes, void* stream);

/* Sets the spin limit, in SM clock cycles, of the bounded device-side waits
 * between the roles of the pipelined kernels (the 3-D sweep's copy producer
 * and its consumers) for every launch that follows, process-wide; 0 restores
 * the default (2e9 cycles, about one second).  Waits by which a kernel that
 * gives up first lets its own copies land keep the default, so a kernel always
 * exits with nothing in flight.  A limit shorter than a copy's latency makes
 * the waits give up: the calls launched with it set the flag that
 * tp_workspace_status reports as TP_ERR_TIMEOUT, their misfit and gradient
 * norm read NaN, and their other results are invalid.  The paper has no
 * counterpart: this exists to exercise the timeout path.  Errors: TP_ERR_ARG
 * (cycles < 0). */
tp_status tp_set_wait_limit(int64_t cycles);

/* Thread-local message of the last error on the calling thread ("" if none). */
const char* tp_last_error(void);

/* ---- kernel timing (CUDA events around every launch, for rooflines) ---- */
typedef enum {
  TP_KERNEL_STENCIL = 0,  /* leapfrog step, forward or adjoint (K1/K2) */
  TP_KERNEL_IMAGING = 1,  /* stencil-form imaging / probe combine sweep */
  TP_KERNEL_PROBE_GEMM = 2, /* windowed probe GEMM on tcgen05 (K3) */
  TP_KERNEL_POINT = 3,    /* source injection + receiver sampling */
  TP_KERNEL_REDUCE = 4,   /* residual, misfit and norm reductions */
  TP_KERNEL_OTHER = 5,    /* setup kernels, probe generation, finish */
  TP_KERNEL_STEP_IMAGING = 6, /* 3-D adjoint step fused with the imaging
                                 condition of the full-storage gradient */
  TP_KERNEL_KINDS = 7
} tp_kernel_kind;

/* Starts recording a CUDA event pair around every kernel launch of the
 * calling process (at most `max_launches` pairs; 0 = 65536). */
tp_status tp_profile_begin(int max_launches);
/* Stops recording, synchronises and writes per kind the summed duration in
 * ms and the number of launches (host arrays of TP_KERNEL_KINDS entries). */
tp_status tp_profile_end(double* ms, int64_t* launches);
/* Name of a tp_kernel_kind. */
const char* tp_kernel_name(int kind);

#ifdef __cplusplus
}
#endif

#endif /* TPROBE_H */
