/*
 * cgks.h -- C-ABI of the GB300 CGKS-5 library: the per-stage sweep of the
 * fifth-order compact gas-kinetic scheme of arXiv 2508.08965 on one GPU.
 *
 * One S2O4 step (temporal discretisation section) runs two stages; each stage
 *   (a) reconstructs, on the standard reference cell (Sec. 4), the quartic
 *       compact polynomial of Eq. (compact-big-ref) from cell averages,
 *       cell-averaged gradients and line-averaged derivatives, blended with
 *       the six linear sub-stencil polynomials by the GENO path function
 *       (Eq. weno-new and the path function of Sec. 3.3);
 *   (b) evaluates the gas-kinetic time-dependent interface solution
 *       (Eq. flux) at the 2x2 (3-D) or 2 (2-D) Gauss points of every face and
 *       takes its moments (Eqs. deri-t-f, deri-t-q);
 *   (c) updates cell averages by S2O4 and cell/line-averaged derivatives from
 *       the evolved interface values (Eqs. derivative, derivative-l).
 *
 * Problem statement: conservative variables Q = (rho, rho U, rho V[, rho W],
 * rho E) of an ideal gas (Sec. 2), E = |U|^2/2 + p/((gamma-1) rho);
 * Navier-Stokes through the collision time tau = mu/p (Sec. 6).
 *
 * State layout (host and device buffers alike): structure of arrays of
 * doubles, state[(f * nv + v) * ncell + cell], cell = i + n0*(j + n1*k),
 * nv = dim + 2 variables and nf = 1 + dim + L fields per variable:
 *   f = 0          cell average,
 *   f = 1..dim     cell-averaged gradient (physical coordinates),
 *   f = 1+dim+s    line-averaged derivative s = axis*gpf + k (gpf = 4 in 3-D,
 *                  2 in 2-D): difference of the values at the paired Gauss
 *                  points k of the cell's two faces normal to `axis`, divided
 *                  by their physical distance (Eq. derivative-l).
 * Gauss point k of a face: tangential axes (a, b) in increasing order,
 * coordinate along a is 1/2 - g for even k and 1/2 + g for odd k, along b
 * 1/2 - g for k < 2 and 1/2 + g otherwise, g = 1/(2 sqrt 3).
 *
 * Conventions: every call returns a cgks_status; on error the message is kept
 * for cgks_last_error.  The caller owns every buffer it passes; the library
 * copies from/to them and owns all device memory it allocates.  Calls on one
 * context are not thread-safe.  All work is queued on the context's stream.
 */
#ifndef CGKS_H
#define CGKS_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CGKS_OK = 0,
  CGKS_EINVAL = -1,      /* invalid argument */
  CGKS_ENOMEM = -2,      /* device allocation failed */
  CGKS_ECUDA = -3,       /* a CUDA runtime call failed */
  CGKS_ENONPHYS = -4,    /* non-positive density/pressure that even chi = 0 cannot cure */
  CGKS_ETIMEOUT = -5,    /* a bounded device wait gave up (the flux kernel's TMA staging) */
  CGKS_ESTATE = -6,      /* call made in the wrong state */
  CGKS_EUNSUPPORTED = -7, /* option the library does not support */
  CGKS_ETOOLARGE = -8     /* problem larger than a fixed-size buffer of the library */
} cgks_status;

/* Boundary kinds, per domain face (the paper names its wall and far-field
   conditions in the cylinder and jet tests without formulas; these are
   ghost-cell readings).  Opposite faces are periodic together or not at all.
   PERIODIC: the mesh wraps.
   OUTFLOW: zero-gradient; the stencil's ghosts copy the boundary cell and the
     boundary face sees the interior Gauss-point state on both sides.
   SLIP_WALL / NOSLIP_WALL (uniform boxes only): ghosts are mirror images --
     the normal momentum (no-slip: all momentum) and derivatives along the
     normal change sign; the face solves the GKS problem against the mirror
     image of the interior Gauss-point state, then passes no mass and no energy
     (adiabatic) and its interface values carry no normal (no-slip: no)
     momentum.
   INFLOW (uniform boxes only): a fixed state, bc_state[face] (conservative:
     rho, rho U, rho V[, rho W], rho E); ghosts hold it with zero gradients and
     the face solves the GKS problem against it (supersonic inflow, or any
     prescribed far state). */
enum {
  CGKS_BC_PERIODIC = 0,
  CGKS_BC_OUTFLOW = 1,
  CGKS_BC_SLIP_WALL = 2,
  CGKS_BC_NOSLIP_WALL = 3,
  CGKS_BC_INFLOW = 4
};

/* Mesh and physics description.  Uniform box when nodes == NULL. */
typedef struct {
  int dim;              /* 2 or 3 */
  int n[3];             /* cells per axis (n[2] ignored in 2-D) */
  const double* nodes;  /* host, (n0+1)(n1+1)[(n2+1)] x dim node coordinates, i fastest,
                           or NULL for the box [lo, hi]; copied */
  double lo[3], hi[3];
  int bc[6];            /* CGKS_BC_* per face (-x,+x,-y,+y,-z,+z); a code outside the
                           list or a periodic face opposite a non-periodic one:
                           CGKS_EINVAL; a wall or inflow with nodes != NULL:
                           CGKS_EUNSUPPORTED */
  double bc_state[6][5]; /* CGKS_BC_INFLOW faces: their fixed conservative state */
  double gamma;         /* specific heat ratio */
  double mu;            /* dynamic viscosity; 0 = inviscid */
  double prandtl;       /* Prandtl number for the heat-flux correction (used when mu > 0) */
  int tau_mode;         /* collision time (Sec. 6): 0 tau = 0; 1 inviscid shock
                           capturing 0.05 dt + 5 |dp|/(sum p) dt; 2 viscous mu/p + 5 |dp|/(sum p) dt */
  double cfl;           /* CFL number (0.5 in the paper) */
  double dt_fixed;      /* > 0: constant time step instead of the CFL rule */
  int linear;           /* 1: linear CGKS-5 (chi = 1) */
  double c_chi;         /* GENO path-function constant C (<= 0: default 100) */
  int precision;        /* 0: FP64 throughout; 1: reconstruction, interface flux,
                           weights and derivative fields in FP32, cell averages
                           (accumulated across the S2O4 stages) and metrics in FP64;
                           2: as 0, with the GKS solve of the interior face Gauss
                           points in paired-FP32 arithmetic (hi + lo floats, about
                           48 bits; exp, erfc, sqrt in FP64); other values:
                           CGKS_EUNSUPPORTED.  Batches take 0 or 1. */
  void* stream;         /* cudaStream_t to queue work on; NULL = default stream */
} cgks_mesh_desc;

typedef struct cgks_ctx cgks_ctx;

/* Allocate the device state and metrics of a mesh; metrics are computed once
   (standard-cell Jacobian J0 of Sec. 4, volumes by the trilinear map of the
   Appendix, face area vectors at the Gauss points, line lengths).  *out is set
   only on success. */
cgks_status cgks_create_mesh(const cgks_mesh_desc* desc, cgks_ctx** out);
void cgks_destroy(cgks_ctx* ctx);

int cgks_num_vars(const cgks_ctx* ctx);    /* nv */
int cgks_num_fields(const cgks_ctx* ctx);  /* nf */
long cgks_num_cells(const cgks_ctx* ctx);

/* How the interface-flux kernel of this context stages each face point's
   Gauss-point states in shared memory (no counterpart in the paper, which
   states no kernel design): 1 = one tensor-memory-accelerator (TMA) tile per
   block of 128 points (Cartesian meshes whose cell count is a multiple of
   128), 0 = one cp.async per value and thread (every other mesh, or the
   environment variable CGKS_FLUX_STAGING=cp.async at cgks_create_mesh).
   Results are the same bit for bit.  A TMA tile that does not arrive within
   its bounded wait (about a second) makes cgks_step return CGKS_ETIMEOUT;
   -1 for a NULL context. */
int cgks_flux_staging(const cgks_ctx* ctx);

/* Copy a full state in (layout above), from host (is_device = 0) or device
   memory, and set the time. */
cgks_status cgks_set_state(cgks_ctx* ctx, const double* src, int is_device, double t);
/* Copy the state out; *t (may be NULL) receives the time.  Synchronises. */
cgks_status cgks_get_state(cgks_ctx* ctx, double* dst, int is_device, double* t);

/* The same two copies, enqueued on the context's stream without waiting,
   so that the copies of one context overlap the steps of another (each on
   its own stream).  Stream order keeps them in sequence with this context's
   steps.  The caller keeps src valid and unmodified, and does not read dst,
   until cgks_sync returns (or a later synchronising call on this context:
   cgks_step, cgks_get_state, cgks_set_state from host memory).  Host
   buffers should be page-locked (cudaHostAlloc, cudaHostRegister); copies
   from or to pageable memory are made synchronously by CUDA.  Sets the time
   to t; cgks_get_state_async does not report it.  A copy error may only
   show at the next synchronising call. */
cgks_status cgks_set_state_async(cgks_ctx* ctx, const double* src, int is_device, double t);
cgks_status cgks_get_state_async(cgks_ctx* ctx, double* dst, int is_device);
/* Wait until everything enqueued on the context's stream has finished. */
cgks_status cgks_sync(cgks_ctx* ctx);

/* Advance nsteps S2O4 steps.  t_end > 0 shortens the last step so that the
   time does not pass t_end (and stops there).  t_out / dt_last may be NULL.
   Returns CGKS_ENONPHYS if a state became non-physical: a Gauss-point or
   interface state that the positivity fallbacks (first order) cannot make
   physical, or a cell average with rho <= 0, p <= 0 or a NaN.  The state and
   time are then those of the last good step of this call: the input of the
   step whose reconstruction or flux failed, or the input of the step whose
   output the next time step found non-physical; the steps after it do no
   work.  A state that is non-physical when the call starts is left as it
   is.  Synchronises once. */
cgks_status cgks_step(cgks_ctx* ctx, int nsteps, double t_end, double* t_out, double* dt_last);

/* The CFL time step of the current state (dt = CFL / max over cells of
   sum_d (|U.n_d| + c)/h_d, capped by CFL h^2/(3 nu)). */
cgks_status cgks_compute_dt(cgks_ctx* ctx, double* dt);

/* Initial data from point values.  For cells [cell0, cell0+ncells) the
   library lists the points it needs (per cell: the 5^dim Gauss points of the
   cell, then its face Gauss points in the order gp = (2*axis+side)*gpf + k)
   into dev_pts (device, ncells*npc*dim doubles); the caller evaluates the
   primitive variables (rho, U, V[, W], p) there and passes them back in
   dev_prims (device, ncells*npc*nv doubles).  Averages come from the Gauss
   rule, gradients and line derivatives from the discrete definitions
   (Eqs. derivative, derivative-l) applied to the point values. */
int cgks_init_points_per_cell(const cgks_ctx* ctx);
cgks_status cgks_init_points(cgks_ctx* ctx, long cell0, long ncells, double* dev_pts);
cgks_status cgks_init_from_prims(cgks_ctx* ctx, long cell0, long ncells, const double* dev_prims);

/* The GENO weight chi of the first stage of the last step, [v][cell]. */
cgks_status cgks_get_chi(cgks_ctx* ctx, double* dst, int is_device);

/* Per-kernel timing with CUDA events on the context stream: enable/disable
   (resets the counters), then read kernel names, launch counts and total
   milliseconds.  names receives up to cap entries; returns the count. */
cgks_status cgks_profile_enable(cgks_ctx* ctx, int on);
int cgks_profile_read(cgks_ctx* ctx, const char** names, long* launches, double* total_ms, int cap);

/* Time step of a state the caller holds on the device, computed without
   allocating any device memory.  The paper has no counterpart: this exists
   for callers that cannot call cudaMalloc -- e.g. an application whose device
   memory is reserved up front by another allocator, or a timed loop that
   must not pay for allocation, which can synchronise the device.
   desc: a uniform box (nodes must be NULL, else CGKS_EUNSUPPORTED) with dim,
   n, lo, hi, gamma, mu, cfl, dt_fixed and stream as for cgks_create_mesh;
   dev_state: pointer to a state in the public layout in memory of the
   current device (else CGKS_EINVAL); only its averages are read; *dt_out
   (host) receives the same dt as cgks_compute_dt would for that state, or
   dt_fixed when that is positive.  A cell whose rate is not finite and
   positive (e.g. negative pressure) gives CGKS_ENONPHYS.  At most
   CGKS_DT_NOALLOC_MAX_CELLS cells, else CGKS_ETOOLARGE before any CUDA call.
   The work space is a fixed array of (CGKS_DT_NOALLOC_MAX_CELLS/256 + 1)
   8-byte words that every GPU loading the library holds until the process
   exits; the first call on a device also looks up that array's device
   address (cudaGetSymbolAddress), so make it before any stream capture.
   Every call overwrites the words it reads, so none has to start at zero.
   All calls share the array: calls whose kernels overlap on the GPU race.
   Synchronises the stream. */
#define CGKS_DT_NOALLOC_MAX_CELLS 16777216
cgks_status cgks_compute_dt_noalloc(const cgks_mesh_desc* desc, const double* dev_state, double* dt_out);

/* The volume averages of the TGV diagnostics (Sec. 6.2) for the current
   state: *ek = (1/(rho0 |Omega|)) sum_cells (1/2) |m|^2/rho |cell| and
   *enstrophy = (1/(rho0 |Omega|)) sum_cells mu |curl U|^2 |cell|, with rho0
   the mean density and the velocity gradient from the cell averages and the
   cell-averaged gradients, d_k U_i = (d_k m_i - U_i d_k rho)/rho (cell-centred
   quadrature, second order; the paper integrates reconstruction
   derivatives).  mu is the mesh's constant viscosity.  Either output may be
   NULL.  Synchronises. */
cgks_status cgks_diagnostics(cgks_ctx* ctx, double* ek, double* enstrophy);

/* Copy the last error message (NUL-terminated, truncated to cap). */
cgks_status cgks_last_error(const cgks_ctx* ctx, char* msg, size_t cap);

/* ---- Batched ensemble ----------------------------------------------------
   Many independent meshes (cases) of uneven size advancing together: one
   launch per kernel and phase covers every case, and a run of nsteps S2O4
   steps is captured once as a CUDA graph and replayed.  The paper has no
   counterpart; each case computes exactly what cgks_step computes for it
   (its own CFL time step, time, boundaries and physics).  Cases are uniform
   boxes (nodes == NULL) of one dim and one precision; their descriptors'
   stream fields are ignored in favour of the batch's stream. */
typedef struct cgks_batch cgks_batch;

/* Launch configuration of the batched kernels.  The reconstruction works on
   tiles of tile_x x tile_y cells of one (i, j) plane (tile_x * tile_y <= 128,
   one thread per cell); the other kernels on tiles of 128 (256 for the time
   step) work items.  *_blocks = 0 launches one block per tile; n > 0 a
   persistent grid of n blocks per SM that walks the tiles. */
typedef struct {
  int tile_x, tile_y;
  int recon_blocks;
  int flux_blocks;   /* also the boundary faces */
  int update_blocks; /* also the time-step reduction */
} cgks_batch_tiles;

/* Validates every descriptor (as cgks_create_mesh, plus: equal dim and
   precision, nodes == NULL else CGKS_EUNSUPPORTED) and allocates all cases'
   arrays.  stream: cudaStream_t for all work (must be non-NULL for graphs
   and tuning).  States start at zero: set each case with
   cgks_batch_set_state. */
cgks_status cgks_batch_create(const cgks_mesh_desc* descs, int ncase, void* stream, cgks_batch** out);
void cgks_batch_destroy(cgks_batch* b);
int cgks_batch_num_cases(const cgks_batch* b);
long cgks_batch_num_cells(const cgks_batch* b);
/* State of case k in the public layout of that case's mesh (as
   cgks_set_state / cgks_get_state). */
cgks_status cgks_batch_set_state(cgks_batch* b, int k, const double* src, int is_device, double t);
cgks_status cgks_batch_get_state(cgks_batch* b, int k, double* dst, int is_device, double* t);
/* Per-case time and last time step into host arrays of ncase (may be NULL). */
cgks_status cgks_batch_times(cgks_batch* b, double* t, double* dt_last);
/* Advance every case nsteps steps.  use_graph = 1: one graph launch (captured
   on first use for this nsteps; changing the tiles drops the graphs);
   0: plain launches.  Synchronises once; CGKS_ENONPHYS if any case became
   non-physical. */
cgks_status cgks_batch_step(cgks_batch* b, int nsteps, int use_graph);
cgks_status cgks_batch_get_tiles(const cgks_batch* b, cgks_batch_tiles* out);
cgks_status cgks_batch_set_tiles(cgks_batch* b, const cgks_batch_tiles* t);
/* Autotuner: times each phase of a stage (reps repetitions) under every
   candidate tile shape and grid size on the batch's current data, keeps the
   fastest per phase and returns it in *chosen (and the sum of the phase times
   in *ms_best, may be NULL).  The cases' states and times are unchanged. */
cgks_status cgks_batch_tune(cgks_batch* b, int reps, cgks_batch_tiles* chosen, double* ms_best);
cgks_status cgks_batch_last_error(const cgks_batch* b, char* msg, size_t cap);

/* ---- Learned troubled-cell selector ---------------------------------------
   Not in the paper (its GENO weights, Sec. 3.3, run on every cell).  A small
   network predicts from 16 normalised stencil features of a cell (face jumps,
   second-difference ratios, line-derivative spread and mismatch, pooled per
   variable class) whether the cell can skip the adaptive weights and take the
   fifth-order polynomial directly (chi = 1 for all its variables).  Inference
   runs inside the reconstruction kernel in BF16 on the tensor cores (weights
   and features rounded to BF16, FP32 sums).  A cell whose logit reaches
   thr_skip skips; below it (low confidence, or a predicted troubled cell) the
   full GENO weights run as without the selector; the positivity fallbacks
   apply either way.
   params (host): CGKS_SEL_NPARAM floats, W1[32][16] b1[32] W2[32][32] b2[32]
   W3[32][32] b3[32] w4[32] b4, row-major [out][in]; NULL switches the
   selector off.  thr_lo <= thr_skip (else CGKS_EINVAL) only splits the
   non-skipped cells into low-confidence (thr_lo < logit) and confident
   troubled cells for the counters. */
#define CGKS_SEL_NFEAT 16
#define CGKS_SEL_NPARAM 2689
cgks_status cgks_set_selector(cgks_ctx* ctx, const float* params, float thr_skip, float thr_lo);
/* Cell reconstructions that skipped, and that ran GENO with low confidence,
   since the selector was set (both stages of every step). */
cgks_status cgks_selector_stats(cgks_ctx* ctx, unsigned long long* skips, unsigned long long* unsure);
/* The 16 features of every cell of the current state into dev_out (device,
   ncell x 16 floats, cell-major): training samples.  Synchronises. */
cgks_status cgks_selector_features(cgks_ctx* ctx, float* dev_out);
cgks_status cgks_batch_set_selector(cgks_batch* b, const float* params, float thr_skip, float thr_lo);
cgks_status cgks_batch_selector_stats(cgks_batch* b, unsigned long long* skips, unsigned long long* unsure);

/* Training arithmetic of the selector network, FP32 on device buffers
   (stream: cudaStream_t or NULL).  Loss: the weighted binary cross-entropy of
   the logits, sum_s w_s (softplus(z_s) - y_s z_s) / sum_s w_s.
   cgks_mlp_loss_grad: X [n][16], labels y and weights w [n] (device); writes
   the gradient (CGKS_SEL_NPARAM floats, device) and *loss_out (host).
   Blocked sums in a fixed order (deterministic); allocates its work space
   stream-ordered and synchronises the stream.
   cgks_mlp_logits: logits [n] (device), FP32 forward pass.
   cgks_mlp_adam: one Adam update of params with first/second moments m, v
   (device, zero before step 1); step counts from 1. */
cgks_status cgks_mlp_loss_grad(const float* dev_params, const float* dev_X, const float* dev_y, const float* dev_w,
                               long n, float* dev_grad, float* loss_out, void* stream);
cgks_status cgks_mlp_logits(const float* dev_params, const float* dev_X, long n, float* dev_out, void* stream);
cgks_status cgks_mlp_adam(float* dev_params, const float* dev_grad, float* dev_m, float* dev_v, int step, float lr,
                          float beta1, float beta2, float eps, void* stream);


#ifdef __cplusplus
}
#endif
#endif
