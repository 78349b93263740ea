/*
 * prs.h -- C ABI of libprs: the Press-Ryden-Spergel (PRS) domain-wall evolution of
 * Correia & Martins, arXiv:1710.10420, on one NVIDIA GB300 (sm_103a).
 *
 * The method (Sec. II of the paper):
 *   Eq. 2  phi'' + alpha (dln a/dln eta) phi'/eta - lap phi = -a^beta dV/dphi,
 *          V(phi) = V0 (phi^2/phi0^2 - 1)^2 (Eq. 1); PRS takes alpha = 3, beta = 0.
 *   Eq. 3  lap phi: nearest-neighbour second difference on a periodic lattice
 *          (5-point in 2D, 7-point in 3D), divided by dx^2.
 *   Eq. 4  dphi^{n+1/2} = [(1-delta) dphi^{n-1/2} + deta (lap phi^n - a^beta dV/dphi^n)]/(1+delta)
 *   Eq. 5  phi^{n+1}    = phi^n + deta dphi^{n+1/2}
 *   Eq. 6  delta_n = alpha deta (dln a/dln eta) / (2 eta_n),  eta_n = eta0 + n deta
 *   Eq. 7  A/V = dA sum_links delta_pm |grad phi|/(|phi,x|+|phi,y|+|phi,z|) / V
 *   Eq. 8  (gamma v)^2 = (1/2N) sum_{wall sites} dphi^2 / V(phi)
 *
 * Conventions for every call:
 *   - Every entry point returns a status code (PRS_OK = 0, negative on error) and
 *     never throws or aborts; prs_strerror() names the code.  On error, output
 *     arguments are left unchanged unless stated otherwise.
 *   - Fields are structure-of-arrays: phi and dphi (= d phi / d eta) each hold
 *     nx*ny*nz values, row-major with x fastest: idx = x + nx*(y + ny*z).
 *     Element type is float (PRS_FP32) or double (PRS_FP64).
 *   - "Host" pointers are ordinary CPU memory (pinned or pageable); "device"
 *     pointers are CUDA global memory of the current device.
 *   - Work is queued on the stream given at creation (NULL = the legacy default
 *     stream).  Calls that return host results synchronise that stream.
 *   - A handle must not be used from two host threads at once.  Calls on different
 *     handles may run concurrently from different host threads (each run has its
 *     own stream; the library keeps no other unsynchronised state), which lets one
 *     run's host transfers overlap another run's kernels.
 */
#ifndef PRS_H
#define PRS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- status codes */
#define PRS_OK 0
#define PRS_EINVAL (-1)     /* bad argument: shape, CFL, precision, NULL handle ... */
#define PRS_ENOMEM (-2)     /* device or host allocation failed                     */
#define PRS_ECUDA (-3)      /* a CUDA runtime call or kernel launch failed          */
#define PRS_ETIMEOUT (-4)   /* a bounded device-side wait gave up                    */
#define PRS_ENONFINITE (-5) /* a diagnostic found non-finite phi or dphi            */
#define PRS_ESTATE (-6)     /* call out of order (e.g. measuring before prs_init)   */

/* ---------------------------------------------------------------- precision */
#define PRS_FP32 0 /* float storage and arithmetic; FP64 diagnostic sums           */
#define PRS_FP64 1 /* double storage and arithmetic                                 */

/* ---------------------------------------------------------------- flags */
/* FP64 only: evaluate each site in the canonical order with no fused multiply-add,
 * so that fields are bit-identical to a sequential IEEE-754 double evaluation of
 * Eqs. 3-5; the diagnostic sums are reduced in a fixed order in every mode. */
#define PRS_REPRO 1u
/* FP32 only (ignored in FP64, where division and square root are always IEEE):
 * evaluate the wall diagnostics (Eqs. 7, 8) with correctly rounded division and
 * square root, as the generic diagnostic kernel does, instead of the fast kernels'
 * hardware reciprocal square root and approximate division.  The leapfrog step has
 * no division or square root: with one step per pass (tblock = 1) the fields are
 * bit-identical with and without the flag (prs_step_measure's diagnostics then run as
 * a separate pass, which can change how later steps group into two-step passes).
 * Sec. III compares single precision with and without correctly rounded divide and
 * square root.
 * prs_step_measure then runs the diagnostics and the steps as separate passes.
 * Ensembles (prs_batch_create) reject it. */
#define PRS_FP32_CR 2u
/* Checks after every call that queues work (slower; for development):
 *   - the run's stream is synchronised, so an asynchronous CUDA error is returned
 *     (PRS_ECUDA) by the call that caused it;
 *   - a bounded device-side wait that gave up is returned at once (PRS_ETIMEOUT);
 *   - library-owned fields are allocated between 4 KiB guard bands holding a byte
 *     pattern; a changed band (a kernel wrote past a field) gives PRS_ECUDA with
 *     "guard band ... overwritten" in prs_last_error();
 *   - after a call that changes the state, phi and dphi are scanned: any non-finite
 *     value gives PRS_ENONFINITE.
 * Bound (caller-owned) buffers get every check but the guard bands. */
#define PRS_DEBUG 4u

/* Observables of prs_adjoint (not in the paper: smooth stand-ins for Eq. 7). */
#define PRS_OBS_GRAD_ENERGY 0 /* J = 1/2 sum_s sum_d ((phi_{s+e_d} - phi_s)/dx)^2            */
#define PRS_OBS_SMOOTH_AREA 1 /* J = 1/(S dx) sum_links (1 - tanh(phi_s/eps) tanh(phi_t/eps))/2 */

typedef struct prs_sim prs_sim;     /* one lattice run; opaque, owned by the library */
typedef struct prs_batch prs_batch; /* an ensemble of independent runs              */

/* Parameters of one run (Eq. 2, Eq. 6, and the lattice).  Configs of the paper's
 * kind use dx = 1, deta = 0.1, eta0 = 1, alpha = 3, beta = 0, phi0 = 1, W0 = 10. */
typedef struct {
    int32_t dims;      /* 2 or 3                                                    */
    int32_t precision; /* PRS_FP32 or PRS_FP64                                      */
    int64_t N;         /* box side along x (and along y, z unless Ny, Nz are set); >= 3 */
    int64_t Ny, Nz;    /* sides along y and z; 0 means N.  Nz is ignored in 2D       */
    double dx;         /* lattice spacing (> 0)                                     */
    double deta;       /* conformal time step (> 0)                                 */
    double eta0;       /* conformal time of step 0 (> 0)                            */
    double alpha;      /* damping coefficient of Eq. 2 (PRS: 3)                     */
    double beta;       /* force exponent of a^beta (PRS: 0); a(eta) = eta^era_m     */
    double era_m;      /* dln a / dln eta: 1 radiation, 2 matter                    */
    double W0;         /* wall thickness: V0 = pi^2/(2 W0^2); +inf gives V0 = 0     */
    double phi0;       /* vacuum value (> 0)                                        */
    uint64_t seed;     /* seed of the random initial field (prs_init with NULL)     */
    uint32_t flags;    /* PRS_REPRO | PRS_FP32_CR | PRS_DEBUG, or 0                 */
    int32_t tblock;    /* leapfrog steps per pass over HBM: 0 = library's choice (FP32
                          3D: 1 below 2^24 sites, else 2 where the two-step tiles get at
                          least 4 rows of y; FP32 2D: 3 on rows of 2048 or more and on
                          boxes of at most 1024 rows, else 2 from 2^24 sites and 1
                          below; otherwise 1; see prs_default_tblock); 2 = two-step passes for FP32 boxes with
                          an x side that is a multiple of 128 (3D; z side >= 3) or a
                          multiple of 128 up to 4096 (2D), else 1; 3 = three-step
                          passes for FP32 3D boxes with an x side that is a multiple
                          of 128, a y side that is a multiple of 8 (at least 16) and
                          a z side >= 3, and for FP32 2D boxes with an x side that is
                          a multiple of 128 up to 4096, else as 2; at most 8 (values
                          above the box's limit act as that limit)                  */
} prs_params;

/* One output record of the wall diagnostics (Eq. 7, Eq. 8). */
typedef struct {
    double area_per_volume; /* A/V of Eq. 7, dA = dx^(D-1), V = sites * dx^D          */
    double gamma_v;         /* sqrt of Eq. 8; 0 when there is no wall site            */
    double sum_w;           /* sum over crossing links of |g|/sum_i|g_i|              */
    double sum_ratio;       /* sum over wall sites (V > 0) of dphi^2 / V(phi)         */
    int64_t n_links;        /* links (s, s+e_d) with (phi_s < 0) != (phi_t < 0)       */
    int64_t n_wall;         /* sites with a nearest neighbour of the opposite sign    */
    int64_t n_vzero;        /* wall sites with V(phi) == 0, left out of Eq. 8         */
    int64_t n_nonfinite;    /* sites where phi or dphi is NaN or infinite             */
    int64_t step;           /* n: the field measured is phi^n, dphi^{n-1/2}           */
    double eta;             /* eta_n = eta0 + n deta                                  */
} prs_diag;

/* ------------------------------------------------------------ single runs */

/* Create a run.  Validates the parameters, including the leapfrog stability
 * limit deta^2 (4 D/dx^2 + max|V''|) < 4 (Eqs. 3-5), and allocates the small
 * device scratch used by the diagnostics.  Field buffers are allocated on the
 * first prs_init/prs_set_state unless prs_bind supplies them.
 * stream: a cudaStream_t, or NULL.  *out receives the handle. */
int prs_create(const prs_params* params, void* stream, prs_sim** out);

/* Use caller-owned device buffers for the fields instead of library memory.
 * d_phi_a and d_phi_b each hold one field (the leapfrog writes phi^{n+1} into the
 * buffer that does not hold phi^n); d_dphi holds dphi and is updated in place.
 * Each must be 16-byte aligned and hold sites * element-size bytes; they stay
 * owned by the caller and must outlive the run.  Must precede prs_init. */
int prs_bind(prs_sim* sim, void* d_phi_a, void* d_phi_b, void* d_dphi);

/* Set the initial state (step 0).  h_phi == NULL: phi_s is drawn on the device
 * from SplitMix64 (Steele, Lea & Flood 2014) at counter idx+1 after params.seed,
 * top 24 bits k, phi = (2k+1) 2^-24 - 1: i.i.d. uniform in (-1,1), exact in FP32
 * (the paper's random initial conditions, Sec. III).  h_dphi == NULL: dphi = 0
 * (the first kick starts from dphi^{-1/2} = dphi_init).  Host arrays are copied. */
int prs_init(prs_sim* sim, const void* h_phi, const void* h_dphi);

/* Queue nsteps (>= 0) leapfrog steps (Eqs. 3-6) on the run's stream; returns
 * without waiting (the call never allocates, so it may be captured into a CUDA graph).
 * Step n uses delta_n, eta_n = eta0 + n deta.  Every step of the call must satisfy the
 * stability limit (checked at both ends, where the force prefactor a^beta is largest),
 * else PRS_EINVAL.  Passes of two or three steps (see prs_params.tblock) read dphi
 * across sites and write it out of place, into a second dphi buffer that prs_init,
 * prs_set_state or prs_set_state_device allocate when the run takes multi-step passes
 * (owned by the run, freed by prs_destroy; if that allocation fails, the steps run one
 * per pass).  A call of nsteps runs nsteps / T passes of T = tblock steps, then (T = 3)
 * one pair if two steps remain, then single steps; when the library chooses the steps per
 * pass (tblock = 0, T = 2) on a box that takes three-step passes, an odd count runs one
 * three-step pass instead of a pair and a single step.  Where dphi ends:
 *   - library-owned buffers (no prs_bind, no PRS_DEBUG): after an odd number of
 *     multi-step passes the two dphi buffers swap roles; every step count keeps all its
 *     passes.  prs_device_state returns the current buffer.
 *   - bound buffers (prs_bind) or PRS_DEBUG: dphi ends in the run's own buffer after
 *     every call.  After an odd number of multi-step passes the first single step brings
 *     dphi home; with no single step to do it, the three-step pass of an odd T = 2 count
 *     runs as a pair and a single step, else the last pair as two single steps (T = 2:
 *     counts 2, 6, 10, ...; T = 3: counts 2, 8, 14, ...), else the last triple as a pair
 *     and a single step (T = 3: counts 3, 9, 15, ...). */
int prs_step(prs_sim* sim, int64_t nsteps);

/* Wall diagnostics of the current state (Eq. 7, Eq. 8), reduced on the device in
 * FP64 in a fixed order, then copied to the host; synchronises the stream.
 * Any output pointer may be NULL.  Returns PRS_ENONFINITE (outputs still written)
 * when some phi or dphi is not finite. */
int prs_measure(prs_sim* sim, double* area_per_volume, double* gamma_v, int64_t* n_links,
                int64_t* n_wall_sites);

/* As prs_measure, filling the whole record. */
int prs_measure_ex(prs_sim* sim, prs_diag* out);

/* prs_step(nsteps) fused with the diagnostics of the state at the start of the call
 * (Eq. 7, Eq. 8 on phi^n, dphi^{n-1/2}): for FP32 boxes of the fast path the first
 * step's pass computes both from one read of the state.  *out receives what
 * prs_measure_ex would have returned before the call (out->step = n).  nsteps = 0
 * only measures.  Synchronises at the end. */
int prs_step_measure(prs_sim* sim, int64_t nsteps, prs_diag* out);

/* Checkpoint: copy the current fields to host arrays (either may be NULL) and the
 * step index to *n (may be NULL).  Synchronises. */
int prs_get_state(prs_sim* sim, void* h_phi, void* h_dphi, int64_t* n);

/* Resume: overwrite the fields from host arrays (both required) and set the step
 * index (>= 0).  Bit-exact round trip with prs_get_state. */
int prs_set_state(prs_sim* sim, const void* h_phi, const void* h_dphi, int64_t n);

/* As prs_set_state, but queued on the run's stream without waiting: the call returns
 * once the copies are issued.  The host arrays must stay valid and unchanged until the
 * stream has passed the copies (any later call that synchronises the run, e.g.
 * prs_step_measure, guarantees it).  From pinned host memory the copies overlap other
 * runs' kernels, so one host thread can upload the next run's state while the current
 * run steps; from pageable memory CUDA may complete them before returning. */
int prs_set_state_async(prs_sim* sim, const void* h_phi, const void* h_dphi, int64_t n);

/* As prs_set_state, from device arrays (both required; current device, the run's
 * layout and precision): the copies are queued on the run's stream without waiting, so
 * the arrays must stay valid and unchanged until the stream has passed them, and work
 * that produced them on another stream must be ordered before the call (e.g. by an
 * event).  A source that already is the run's current buffer is left in place. */
int prs_set_state_device(prs_sim* sim, const void* d_phi, const void* d_dphi, int64_t n);

/* Change the conformal time step from the current step n on (the physical equations,
 * alpha = beta = 2, stiffen as a^beta grows: a fixed deta that is stable early fails the
 * stability limit later).  Conformal time continues from the current eta_n:
 * eta_m = eta_n + (m - n) deta for the following steps (params.eta0 is re-based to
 * eta_n - n deta; diagnostics report eta_m).  The kick of the first step with the new
 * deta starts from the stored dphi^{n-1/2} of the old step, as the scheme of Eqs. 4-5
 * does at every step.  PRS_EINVAL if deta <= 0 or if a step of deta at eta_n is unstable
 * or has delta >= 1.  Takes effect for the next queued step (no synchronisation). */
int prs_set_deta(prs_sim* sim, double deta);

/* The largest stable time step at conformal time eta for these parameters:
 * 2 / sqrt(4D/dx^2 + 2 cV(eta) phi0^2), cV(eta) = 4 V0 a(eta)^beta / phi0^2, a = eta^era_m
 * (the leapfrog's limit for the stiffest lattice mode, with the force's slope at its largest
 * for |phi| <= phi0, 2 cV).  A field that overshoots the vacua is stiffer (slope
 * cV (3 phi^2/phi0^2 - 1)): the physical equations (beta = 2), whose walls thin below the
 * lattice spacing, overshoot by tens of per cent, so a schedule should keep a margin (half
 * of this value carries a 2D run with W0 = 8 to eta = 100). */
int prs_stable_deta(const prs_params* params, double eta, double* deta_max);

/* Device pointers of the current fields and the step index (any output may be
 * NULL).  The pointers stay valid until the next prs_step or prs_destroy (a run with
 * library-owned buffers may hold dphi in either of its two dphi buffers). */
int prs_device_state(prs_sim* sim, void** d_phi, void** d_dphi, int64_t* n);

/* Wall diagnostics without any device allocation.  The paper has no counterpart:
 * this exists for callers that cannot let a library call cudaMalloc, e.g. an
 * application that owns every device allocation through its own pool or budget,
 * or a latency-critical loop where cudaMalloc's device-wide synchronisation is
 * not acceptable.  It computes the same record as prs_measure_ex for the fields
 * d_phi, d_dphi (caller-owned device memory, layout and precision of *params)
 * using scratch held in a fixed array compiled into the library: 3 MiB of device
 * memory on every GPU that loads it, kept until the process exits.  Limit:
 * 2^30 sites (1024^3); larger lattices return PRS_EINVAL (see prs_last_error).
 * The first call on a device looks up that array's address with the device
 * current (cudaGetSymbolAddress) and caches it for the life of the process; make
 * that first call before any stream capture, and do not call this entry point after
 * a cudaDeviceReset (the cached address would be stale).  Every call shares the one array, which keeps the last call's
 * contents (the call clears what must start at zero), so calls that overlap on
 * the GPU, from several streams or threads, race: serialise them.  Synchronises
 * `stream`.  out->step is -1 and out->eta 0: the fields carry no step index. */
int prs_measure_noalloc(const prs_params* params, const void* d_phi, const void* d_dphi, void* stream,
                        prs_diag* out);

/* Release the run and the memory the library allocated for it (not bound buffers). */
int prs_destroy(prs_sim* sim);

/* --------------------------------------------------------------- ensembles
 * Many independent runs (the paper's sets of realisations, Sec. III) advanced by
 * one persistent kernel: every run is cut into tiles and the work items
 * (run, tile, step) are taken in an order in which each item only waits, with a
 * bounded spin, for items already taken; diagnostics are fused into the steps
 * that read the same state.  Runs must be FP32 with an x side that is a multiple
 * of 128 dividing 4096 (3D: at most 1024) and 4096/x dividing the y side. */

/* Create an ensemble of nruns runs (each validated as by prs_create), allocate all
 * fields, pick a tile length for each geometry class of runs (4 to 32 planes or bands)
 * and the L2 grouping by timing short trials on them (the autotuner), then set every
 * run to its seeded random initial condition (step 0).  A run that the library steps
 * with multi-step passes (prs_default_tblock >= 2) and whose box has 2^22 sites or more
 * (it fills the GPU by itself), or, in 2D, 2^20 sites or more in rows of at least 1024
 * columns with at least 8 runs of that box in the ensemble (their passes are launched
 * together), is stepped alone, after the persistent launch of the others, as
 * prs_step_measure would step it (its fields and outputs are those of the same run
 * stepped alone; the run holds a second dphi buffer like a prs_sim).  stream may be
 * NULL (the ensemble then creates its own stream). */
int prs_batch_create(const prs_params* runs, int nruns, void* stream, prs_batch** out);

/* Advance run r by nsteps_per_run[r] (>= 0) steps: one persistent launch for the runs
 * it holds, then the runs stepped alone, all on the ensemble's stream.  With
 * measure_every > 0, the diagnostics of run r at its steps n, n+m, ... (n its
 * step at the call, up to n + nsteps_per_run[r]) are written to
 *   out_series[(r*out_capacity + k)*4 + {0,1,2,3}] = {step, A/V, gamma v, n_links}
 * (FP64 reduction, Eq. 7 and Eq. 8); out_capacity must be at least
 * nsteps_per_run[r]/measure_every + 1 for every run.  Synchronises.  Returns
 * PRS_ETIMEOUT if a bounded wait in the kernel gave up (the fields are then not
 * trustworthy). */
int prs_batch_run(prs_batch* batch, const int64_t* nsteps_per_run, int64_t measure_every, double* out_series,
                  int64_t out_capacity);

/* Host copies of run `run`'s fields (either may be NULL) and its step index. */
int prs_batch_get_state(prs_batch* batch, int run, void* h_phi, void* h_dphi, int64_t* n);

/* Overwrite run `run`'s fields from host arrays and set its step index. */
int prs_batch_set_state(prs_batch* batch, int run, const void* h_phi, const void* h_dphi, int64_t n);

/* The autotuner's choice: tile length of `run` (bands of 4096/x rows in 2D,
 * z-planes in 3D; 0 for a run stepped alone) and the bytes of fields per L2 group. */
int prs_batch_tuning(prs_batch* batch, int run, int* tile_len, double* group_bytes);

/* Release the ensemble and everything it allocated. */
int prs_batch_destroy(prs_batch* batch);

/* ---------------------------------------------------------------- adjoint
 * Not in the paper: gradients of a smooth stand-in for the wall diagnostics
 * (PRS_OBS_GRAD_ENERGY or PRS_OBS_SMOOTH_AREA with smoothing width eps_smooth),
 * by the hand-written transpose of the leapfrog step of Eqs. 3-6. */

/* J of the current field (FP64 reduction); synchronises. */
int prs_observable(prs_sim* sim, int observable, double eps_smooth, double* J);

/* Advance the run by nsteps (like prs_step) and return J of the final field with
 * its gradient with respect to the state at the start of the call and to alpha:
 *   *J, *dJ_dalpha (host, FP64);
 *   d_dJ_dphi_init, d_dJ_dv_init: caller-owned device arrays of the run's layout and
 *   precision (either may be NULL), receiving dJ/dphi and dJ/d(dphi) at the start.
 * Memory: with ckpt_every = K > 0, a checkpoint of (phi, dphi) every K steps plus
 * K-1 states of one segment, each segment recomputed from its checkpoint before it
 * is swept backwards; with ckpt_every = 0, every state when nsteps+1 states fit in
 * free device memory (no recomputation), else K = 64.  This working memory stays
 * with the run for the next call (grown when a call needs more) and is released by
 * prs_destroy.  Reverse step n, with lt = lv' + deta lphi':
 *   lphi = lphi' + c2 (L lt - f'(phi) lt),  lv = c1 lt,
 *   dJ/dalpha += sum lt (dc1/dalpha dphi + dc2/dalpha (L phi - f(phi))).
 * On return the run holds the state at step n+nsteps.  Synchronises. */
int prs_adjoint(prs_sim* sim, int64_t nsteps, int observable, double eps_smooth, int64_t ckpt_every, double* J,
                double* dJ_dalpha, void* d_dJ_dphi_init, void* d_dJ_dv_init);

/* Where the time of the last successful prs_adjoint call on this run went, in
 * milliseconds, from CUDA events recorded on the run's stream: ms[0] the forward pass
 * (with its checkpoints or stored states, and J), ms[1] the recomputation of the
 * segments' states, ms[2] the reverse sweep (the reverse steps).  PRS_ESTATE before any
 * such call. */
int prs_adjoint_timing(prs_sim* sim, double ms[3]);

/* Step-n coefficients as the library computes them on the host in FP64:
 * out[0] = c1 = (1-delta_n)/(1+delta_n), out[1] = c2 = deta/(1+delta_n) (Eq. 4, 6),
 * out[2] = cV = 4 V0 a_n^beta / phi0^2 (force prefactor), out[3] = delta_n,
 * out[4] = d delta_n / d alpha. */
int prs_coefficients(const prs_params* params, int64_t n, double out[5]);

/* Leapfrog steps the library fuses into one pass over HBM for these parameters
 * when params->tblock is 0 (>= 1), or a negative status for invalid parameters. */
int prs_default_tblock(const prs_params* params);

/* The most leapfrog steps one pass over HBM can fuse for these parameters (>= 1; a
 * params->tblock above it acts as it): 3 for FP32 2D and 3D boxes the three-step passes
 * take, 2 for the other boxes of the two-step passes, else 1; or a negative status for invalid
 * parameters.  Follows the fusion of Eqs. 3-5 over several steps, which the paper does
 * not do (it launches one kernel per equation and step, Sec. III). */
int prs_max_tblock(const prs_params* params);

/* Self-test of failure detection (no counterpart in the paper).  Launches one
 * CTA that waits on an mbarrier phase that can never complete (the bounded wait
 * of the library's kernels, limit 2 s) and spins on a flag nothing sets (limit
 * 0.2 s).  Both waits must give up; the call then returns PRS_ETIMEOUT, with the
 * CUDA context still usable, and the error bits seen in *codes (may be NULL). */
int prs_selftest_wait_timeout(void* stream, unsigned int* codes);

/* Human-readable name of a status code (static string). */
const char* prs_strerror(int status);

/* Text of the last error the library recorded on this thread: a failed CUDA call,
 * a bounded wait that gave up, or a PRS_DEBUG check (static buffer). */
const char* prs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PRS_H */
