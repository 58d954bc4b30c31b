/*
 * etd.h - C ABI of the GB300 (sm_103a) exponential-integrator Q1 finite-element solver.
 *
 * Problem (Section 1, eq. (1.1); Section 2, eq. (2.1)): u_t = D Lap u + f(u) on a rectangle in 2D or
 * 3D with homogeneous Dirichlet data or periodic boundary conditions (Section 4, closing remarks),
 * f(u) = flin u + fcub u^3 + flog artanh(u) (Allen-Cahn: flin = 1, fcub = -1, flog = 0; the
 * Flory-Huggins reaction of Example 5.3, (theta/2) ln((1-u)/(1+u)) + theta_c u: flin = theta_c,
 * fcub = 0, flog = -theta), applied to nodal values (the tensor F of Section 4 read as F = M f(U)).
 * Space: Q1 (multilinear) elements on a uniform mesh with N_a intervals of size h_a per axis
 * (Section 2.1); the unknowns are the (N_x-1)(N_y-1)[(N_z-1)] interior nodal values.
 * Time: one EIFE1 step, eq. (2.13) (ETDRK1), or one EIFE2 step, eq. (2.14) with c_1 = 0 and
 * c_2 in (0, 1] (ETDRK2; the paper's experiments use c_2 = 1/2, Section 5).
 * Fast solve (Section 4): A_a = (h_a/6) R and B_a = (1/h_a) G^D share the orthonormal sine basis
 * S_a = sqrt(2/N_a) sin(i j pi / N_a), so each step is a forward DST-I along every axis, a per-mode
 * scaling by phi-functions of -tau D (mu_x,i + mu_y,j [+ mu_z,k]) with
 * mu_a,i = (6/h_a^2)(1 - cos(i pi/N_a))/(2 + cos(i pi/N_a)), and inverse DST-I along every axis.
 * Periodic: A_a = (h_a/6) circ(4, 1, .., 1) and B_a = (1/h_a) G^P are circulant with eigenvalues
 * depending on cos(2 pi i/N_a) only, so the orthonormal discrete Hartley transform
 * H_a = N_a^{-1/2} cas(2 pi i j/N_a) (cas = cos + sin; symmetric, H^2 = I) diagonalises them and takes
 * the place of the per-axis DFT / inverse DFT of Section 4, with
 * mu_a,i = (6/h_a^2)(1 - cos(2 pi i/N_a))/(2 + cos(2 pi i/N_a)), i = 0..N_a-1.
 *
 * Conventions for every entry point:
 *  - A field `u` is the array of interior nodal values, x fastest (C order
 *    [N_z-1][N_y-1][N_x-1] or [N_y-1][N_x-1]), dense, element type per etd_options.dtype; on a
 *    periodic plan every node 0..N_a-1 is an unknown ([N_z][N_y][N_x] or [N_y][N_x]).
 *  - Device pointers are CUDA device (or managed) memory owned by the caller; the plan never frees
 *    them. `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Calls enqueue work asynchronously on `stream` unless stated; they return before the GPU work
 *    completes. Errors found on the host are returned before any GPU work is enqueued.
 *  - No call aborts, traps or exits. Every call returns an etd_status; etd_last_error() gives a
 *    human-readable detail for the calling thread's most recent failure.
 *  - A plan is not thread-safe: use one plan per host thread, or serialise calls.
 */
#ifndef ETD_GB300_H
#define ETD_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct etd_plan_s* etd_plan;   /* opaque; owned by the library, released by etd_destroy */

typedef enum {
  ETD_OK = 0,
  ETD_ERR_INVALID_ARG = 1,   /* a contract violation detected on the host; nothing was enqueued */
  ETD_ERR_UNSUPPORTED = 2,   /* valid request the library cannot run (e.g. an axis length it has no kernel for) */
  ETD_ERR_CUDA = 3,          /* a CUDA runtime call failed; see etd_last_error() */
  ETD_ERR_OOM = 4,           /* device or pinned-host allocation failed */
  ETD_ERR_NONFINITE = 5,     /* etd_monitor found NaN/Inf values in the field */
  ETD_ERR_TIMEOUT = 6        /* a tensor-core pass gave up waiting for its own pipeline (a lost
                                arrival; its CTAs exit instead of hanging) and the field is invalid;
                                reported by the next synchronising call (etd_run_host, etd_monitor) */
} etd_status;

typedef enum { ETD_ETDRK1 = 1, ETD_ETDRK2 = 2 } etd_scheme;   /* EIFE1 eq. (2.13), EIFE2 eq. (2.14) */
typedef enum { ETD_F64 = 0, ETD_F32 = 1 } etd_dtype;            /* arithmetic and storage type of u */
/* Transform implementation of the DST-I along each axis.
 * ETD_ROUTE_FFT: FP32 uses the odd extension (a length-2N complex FFT per pair of pencils; rounding
 *   grows like log N); FP64 uses the half-length recurrence below.
 * ETD_ROUTE_FFT_HALF: a length-N complex FFT per pair of pencils followed by a prefix sum (half the
 *   work; rounding grows like sqrt(N/2) eps).
 * ETD_ROUTE_AUTO: per axis, FP32 takes ETD_ROUTE_FFT for N >= 512 and ETD_ROUTE_FFT_HALF below;
 *   FP64 always takes the recurrence.
 * ETD_ROUTE_FFT_SPLIT (FP32; otherwise as ETD_ROUTE_AUTO): Dirichlet axes of N = 1024 (strided ones when
 *   N[0] is a multiple of 4) run a split-radix DST-I: the odd outputs are a DST-III of length N/2, the
 *   even ones split once more into a DST-III of length N/4 and a DST-I of length N/4, each computed by a
 *   complex FFT that fits in one warp (512, 256 and 512 points per pair of pencils against 2048 for the
 *   odd extension; rounding grows like log N, and is smaller than the odd extension's in practice).
 *   Exact arithmetic equal to the other FFT routes; batches take it as ETD_ROUTE_AUTO.
 * FP32 2D plans on the FFT routes take the phi-function weights of the stage combinations from per-mode
 * tables of FP64 values rounded once to FP32 (12 bytes per unknown for EIFE2, 4 for EIFE1, up to 64 MiB;
 * larger and 3D plans evaluate them per mode in FP32).
 * ETD_ROUTE_GEMM_TF32 and ETD_ROUTE_GEMM_BF16X3 (FP32 plans only; every N[a] a multiple of 32):
 *   the DST-I along an axis is the dense product with the N x N sine matrix S_a of Section 4 (periodic
 *   plans: the N x N orthonormal Hartley matrix),
 *   computed on the tensor cores with FP32 accumulation and written transposed, so each pass
 *   contracts a contiguous axis. TF32: the field's values enter the product with TF32 precision
 *   (10 stored mantissa bits), S_a is rounded to TF32. BF16X3: both operands are split into bf16
 *   high and low parts and hi*hi + hi*lo + lo*hi are accumulated (about 16 significant bits per
 *   operand). Errors against the FP64 solution are far above the FFT routes' (see the route's
 *   documented tolerance); the state between steps is spectral along every axis. */
typedef enum {
  ETD_ROUTE_AUTO = 0,
  ETD_ROUTE_FFT = 1,
  ETD_ROUTE_FFT_HALF = 2,
  ETD_ROUTE_GEMM_TF32 = 3,
  ETD_ROUTE_GEMM_BF16X3 = 4,
  ETD_ROUTE_FFT_SPLIT = 5
} etd_route;

typedef struct {
  etd_dtype dtype;   /* default ETD_F64 */
  etd_route route;   /* default ETD_ROUTE_AUTO (the DST-I by FFT kernels) */
  double c2;         /* EIFE2 stage node c_2 in (0, 1]; default 0.5 (Section 5) */
  double flin;       /* f(u) = flin*u + fcub*u^3 + flog*artanh(u); defaults 1, -1, 0 (Allen-Cahn) */
  double fcub;
  int debug;         /* default 0. ETD_DEBUG_STALL_FIRST_GEMM_PASS (GEMM routes): the first tensor-core
                        pass of every etd_run withholds its accumulator-ready signal, so that pass's
                        epilogue warps wait out their 2 s limit, abort and set the plan's error word;
                        the next synchronising call returns ETD_ERR_TIMEOUT and that run's field is
                        invalid. Tests the failure path. ETD_DEBUG_BATCH_SERIAL / ETD_DEBUG_BATCH_PARALLEL
                        (batches): take that steady-state schedule instead of timing both at creation.
                        Any other value is ignored. */
  int bc;            /* boundary condition of every axis: ETD_BC_DIRICHLET (default) or ETD_BC_PERIODIC */
  double flog;       /* coefficient of artanh(u) = (1/2) ln((1+u)/(1-u)) in f; default 0. Nonzero values
                        run on periodic plans and batches (any route) and on the GEMM routes; a Dirichlet
                        plan on an FFT route or a Dirichlet batch returns ETD_ERR_UNSUPPORTED. Where it is nonzero the
                        field must stay in (-1, 1) (|u| >= 1 gives non-finite values, which
                        etd_monitor reports). */
} etd_options;
#define ETD_DEBUG_STALL_FIRST_GEMM_PASS 0x5A11
#define ETD_DEBUG_BATCH_SERIAL 0x5A12
#define ETD_DEBUG_BATCH_PARALLEL 0x5A13
#define ETD_BC_DIRICHLET 0
#define ETD_BC_PERIODIC 1

/* Fill *opt with the defaults above. Returns ETD_ERR_INVALID_ARG if opt is NULL. */
etd_status etd_options_default(etd_options* opt);

/*
 * Create a plan for `ndim` in {2, 3} axes with N[a] intervals (N[0] = N_x, the fastest axis) of
 * size h[a] > 0, diffusion D > 0 and time step tau > 0 (Section 2.2, uniform tau_n = tau).
 * Allocates the device workspace (six fields of N_x*N_y[*N_z] elements on the FFT routes, five on the
 * GEMM routes and where the last axis runs the split-radix kernels) and the FP64-derived
 * tables (eigenvalues mu_a, exp(-tau D mu_a), exp(-c2 tau D mu_a), twiddles) on the current
 * device, and uploads them. Supported N[a]: 2^k (4..2048) and 3*2^k (6..1536).
 * Periodic plans (opt->bc = ETD_BC_PERIODIC) run the Hartley kernels on every FFT route (AUTO,
 * FFT and FFT_HALF are the same there: one length-N complex FFT per pair of pencils), and the
 * Hartley matrix on the GEMM routes.
 * opt may be NULL (defaults). On success *out receives the plan.
 * Errors: ETD_ERR_INVALID_ARG (out/N/h NULL, ndim not 2 or 3, N[a] < 2 or odd, h <= 0, D <= 0,
 * tau <= 0, c2 outside (0, 1], non-finite values, unknown route or bc, a GEMM route with dtype
 * ETD_F64), ETD_ERR_UNSUPPORTED (N[a] without a kernel; a GEMM route with N[a] not a multiple of
 * 32; flog != 0 on a Dirichlet plan of an FFT route), ETD_ERR_OOM, ETD_ERR_CUDA.
 */
etd_status etd_plan_create(etd_plan* out, int ndim, const int64_t* N, const double* h, double D,
                           double tau, etd_scheme scheme, const etd_options* opt);

/* Advance the device field u (in place) by `nsteps` >= 0 time steps on `stream`. nsteps = 0 is a
 * no-op. Equivalent to nsteps calls of etd_step up to rounding (the internal state between steps
 * stays spectral along all axes but the last, or all axes on the GEMM routes). Errors: ETD_ERR_INVALID_ARG (plan or u NULL,
 * nsteps < 0), ETD_ERR_CUDA.
 * Runs (plans and batches) replay steady-state steps from a CUDA graph of ETD_GRAPH_STEPS time steps
 * (environment variable, default 32; 0: every step as direct launches), and pass kernels launch with
 * programmatic dependent launch unless ETD_PDL=0. Both change only timing, not results. */
etd_status etd_run(etd_plan plan, void* u, int64_t nsteps, void* stream);

/* One time step: etd_run(plan, u, 1, stream). */
etd_status etd_step(etd_plan plan, void* u, void* stream);

/* Time-dependent reaction (the scheme of Section 2 takes f = f(t, u); Example 5.1 of Section 5 is of
 * this form): adds a separable source to the reaction,
 *   f(t, u) = flin u + fcub u^3 + amp exp(-rate t) gx[i] gy[j] (gz[k]),
 * gx, gy (and gz in 3D; NULL in 2D) HOST arrays of the N_a - 1 interior nodal values per axis
 * (periodic plans: the N_a nodal values), copied. The source joins the reaction in the pass that
 * transforms it along x, as amp exp(-rate t) (S_x gx) gy (gz) (periodic: H_x gx), evaluated at the
 * stage times of the scheme (t_n for EIFE1 and
 * the first EIFE2 stage, t_n + c2 tau for the second). All profiles NULL removes the source. Synchronous.
 * Errors: ETD_ERR_INVALID_ARG (a missing or extra profile, non-finite values), ETD_ERR_UNSUPPORTED
 * (GEMM routes). */
etd_status etd_set_source(etd_plan plan, double amp, double rate, const double* gx, const double* gy,
                          const double* gz);

/* etd_run starting at time t0 (t_n = t0 + n tau; only a source set with etd_set_source depends on
 * t). etd_run is etd_run_from with t0 = 0. */
etd_status etd_run_from(etd_plan plan, void* u, int64_t nsteps, double t0, void* stream);

/* Nonhomogeneous Dirichlet data (Section 4: the given boundary values of the solution enter the
 * scheme as part of f; Example 5.2 of Section 5). The Galerkin system on all nodes with the boundary
 * nodal values g(t) prescribed has the interior rows
 *   M_II U' + K_II U = M_II f(U) + b(t),  b(t) = M_IB (f(g) - g'(t)) - K_IB g(t)
 * (the reaction taken on nodal values of every node: flin g + fcub g^3 at the boundary nodes; a source
 * set with etd_set_source is defined by its interior profiles and does not enter b), so each stage adds
 * M_II^{-1} b(t) to the nodal
 * reaction: b is assembled on the GPU from the boundary values by the Q1 stencils, transformed along
 * every axis, scaled by the inverse mass eigenvalues and transformed back along the last axis.
 * `fn` supplies the data: fn(t, g, gdot, ctx) writes the boundary values and their time derivatives
 * at time t into the HOST arrays g[count] and gdot[count] (count from etd_boundary_count) and returns
 * 0 (nonzero aborts the run with ETD_ERR_INVALID_ARG). Layout, faces in the order x = 0, x = L_x,
 * y = 0, y = L_y (, z = 0, z = L_z), each over all its nodes including edges and corners, x fastest
 * within a face: 3D x-faces [N_z+1][N_y+1], y-faces [N_z+1][N_x+1], z-faces [N_y+1][N_x+1]; 2D
 * x-faces [N_y+1], y-faces [N_x+1]. A node on several faces takes its value from the first of them
 * in that order. The run calls fn at every stage time (t_n, and t_n + c2 tau for EIFE2), copies the
 * arrays to the device and synchronises `stream` once per time step (no CUDA graph), so such runs
 * are for accuracy, not speed. fn NULL removes the data (homogeneous Dirichlet again).
 * Errors: ETD_ERR_INVALID_ARG (periodic plan), ETD_ERR_UNSUPPORTED (GEMM routes), ETD_ERR_OOM. */
typedef int (*etd_boundary_fn)(double t, double* g, double* gdot, void* ctx);
etd_status etd_set_boundary(etd_plan plan, etd_boundary_fn fn, void* ctx);

/* Number of boundary nodal values per array of the layout above: 2D 2(N_y+1) + 2(N_x+1); 3D
 * 2(N_z+1)(N_y+1) + 2(N_z+1)(N_x+1) + 2(N_y+1)(N_x+1). Errors: ETD_ERR_INVALID_ARG (NULL argument or a
 * periodic plan). */
etd_status etd_boundary_count(etd_plan plan, int64_t* count);

/* Same as etd_run, but u_host is HOST memory (pinned or pageable) of the field's size: the call
 * copies it to a plan-owned device buffer, runs, copies the result back and synchronises the
 * stream before returning. */
etd_status etd_run_host(etd_plan plan, void* u_host, int64_t nsteps, void* stream);

/* Apply the orthonormal DST-I S_a (periodic plans: the orthonormal DHT H_a) along paper axis `axis`
 * (0 = x, 1 = y, 2 = z) to the dense device field `in`, writing the dense device field `out` (may
 * equal `in`). S_a and H_a are symmetric and their own inverses, so this is both the forward
 * transform U~ = S^T (x)_a U of Section 4 and its inverse.
 * Runs the FFT kernels of the plan's dtype on every route (a GEMM-route plan transforms with the FFT
 * variant that ETD_ROUTE_AUTO would take). */
etd_status etd_apply_dst(etd_plan plan, int axis, const void* in, void* out, void* stream);

typedef struct {
  double mass;       /* 1^T M U with M the Q1 mass matrix */
  double energy;     /* 1/2 U^T K U + sum_nodes prod(h) G(u): G(u) = (u^2 - 1)^2 / 4 when flog = 0;
                        otherwise the potential with G' = -f, G(0) = 0,
                        G(u) = -flog (u artanh u + ln(1 - u^2)/2) - flin u^2/2 - fcub u^4/4, which for
                        the Flory-Huggins coefficients is the energy density of Example 5.3,
                        (theta/2)((1+u) ln(1+u) + (1-u) ln(1-u)) - (theta_c/2) u^2 */
  double maxabs;     /* max |u| */
  int64_t nonfinite; /* number of NaN/Inf values */
} etd_monitors;

/* FP64 reductions over the device field u (the plan's boundary condition and reaction); synchronises
 * `stream` and writes *out. Returns ETD_ERR_NONFINITE (with *out filled) when u holds NaN or Inf
 * values. */
etd_status etd_monitor(etd_plan plan, const void* u, etd_monitors* out, void* stream);

/* Kernel-level timing of one etd_run: records CUDA events around every kernel launch, runs
 * `nsteps` steps on `stream`, synchronises, and writes per pass kind the summed duration in
 * milliseconds and the launch count (arrays of length ETD_NUM_PASS_KINDS). Not for production
 * use: the events add launch overhead. Plans with nonhomogeneous Dirichlet data return
 * ETD_ERR_UNSUPPORTED. */
#define ETD_NUM_PASS_KINDS 9
etd_status etd_run_profiled(etd_plan plan, void* u, int64_t nsteps, void* stream,
                            double* ms_per_kind, int64_t* launches_per_kind);

typedef struct {
  int ndim;
  int64_t N[3];
  int64_t unknowns;            /* prod (N_a - 1); periodic: prod N_a */
  int64_t workspace_bytes;     /* device bytes owned by the plan */
  int kernels_per_step;        /* kernel launches per time step in etd_run */
  double bytes_per_step;       /* algorithmic HBM bytes per time step (field passes x size) */
  int dtype;
  int scheme;
} etd_plan_info;

/* Describe a plan. */
etd_status etd_get_plan_info(etd_plan plan, etd_plan_info* info);

/* The phi-function weights of the stage combinations (eqs. (2.13)/(2.14); phi_k of Section 2.2) as the
 * FFT pass kernels evaluate them per mode, in the arithmetic of dtype: for each of the n modes, from
 * zeta[i] = tau lambda_i >= 0, E[i] = e^{-zeta} and Ec[i] = e^{-c2 zeta} (HOST arrays, rounded to dtype
 * on the device as the kernels' tables hold them), writes out[3i] = phi_1(-zeta), out[3i+1] =
 * phi_2(-zeta), out[3i+2] = c2 phi_1(-c2 zeta) (HOST array of 3n doubles). These are the weights of 3D
 * plans and of 2D plans above the per-mode table size; 2D FP32 plans otherwise use FP64 values rounded
 * once. For checking their accuracy; allocates a temporary device buffer and synchronises. Errors:
 * ETD_ERR_INVALID_ARG for NULL arrays (n > 0), n < 0, c2 outside (0, 1], negative or non-finite zeta,
 * non-finite E or Ec. */
etd_status etd_phi_weights(etd_dtype dtype, int64_t n, const double* zeta, const double* E, const double* Ec,
                           double c2, double* out);

/* Name of pass kind k (0 <= k < ETD_NUM_PASS_KINDS), or NULL. */
const char* etd_pass_kind_name(int k);

/* Field monitors without a plan and without allocating (the paper has no counterpart; this serves
 * callers that cannot allocate GPU memory: code running under a framework that owns every
 * allocation or a fixed memory budget, real-time loops where an allocation and the synchronisation
 * it may imply are not allowed, or a health check that must work before any plan exists).
 * Computes the same mass, energy, max|u| and non-finite count as etd_monitor for the dense device
 * field u (ndim in {2, 3}, N[a] intervals of size h[a] per axis, homogeneous Dirichlet, the
 * Allen-Cahn potential (u^2 - 1)^2 / 4, diffusion D, dtype) and writes
 * them to out_dev, a DEVICE pointer to one etd_monitors, asynchronously on `stream`; it does not
 * synchronise and never returns ETD_ERR_NONFINITE (read out_dev->nonfinite instead).
 * Scratch: a fixed array inside this library (partial sums of one CTA per 2048 unknowns), present
 * on every GPU that loads the library until the process exits; at most
 * ETD_MONITOR_NOALLOC_MAX_UNKNOWNS unknowns, larger fields return ETD_ERR_INVALID_ARG. The first
 * call on each device looks the scratch address up (cudaGetSymbolAddress): make that first call
 * before any stream capture on that device. Every call shares the scratch and overwrites all of it
 * that it reads, so calls whose GPU work overlaps (concurrent streams, several host threads) race;
 * serialise them. Calls no allocating routine. */
#define ETD_MONITOR_NOALLOC_MAX_UNKNOWNS 33554432
etd_status etd_monitor_noalloc(int ndim, const int64_t* N, const double* h, double D, etd_dtype dtype,
                               const void* u, etd_monitors* out_dev, void* stream);

/* Release the plan's device memory and graphs. NULL is accepted. */
etd_status etd_destroy(etd_plan plan);

/*
 * Batches of independent 2D problems (same scheme, tau and options; per problem its own mesh and
 * D): many EIFE1/EIFE2 solves (eqs. (2.13)/(2.14)) advanced together. Problem i has N[2i], N[2i+1]
 * intervals of size h[2i], h[2i+1] and diffusion D[i]; the same length rules as etd_plan_create.
 * Each pass of a time step is one kernel launch per distinct length of the transformed axis,
 * covering every problem with that length; the tile size of each launch is tuned at creation by
 * timing the candidates (set ETD_AUTOTUNE=0 to take a fixed choice). Steady-state steps replay as a
 * CUDA graph in one of two schedules: the launches of a pass one after another on one stream, each
 * overlapping its predecessor's tail (programmatic dependent launch), or as parallel graph branches
 * (they cover disjoint problems) joined before the next pass. Creation times both graphs on the
 * workspace and keeps the faster (etd_batch_schedule reports the choice and both times); with
 * ETD_AUTOTUNE=0 the serial schedule is taken. Results equal those of one plan per problem with the same options up to rounding
 * (the batched kernel is a separate instantiation, so the compiler may contract and order the
 * floating-point operations differently; measured differences are at the dtype's rounding level).
 * Allocates per-problem fields and tables on the current device. Errors as for etd_plan_create;
 * count <= 0 is ETD_ERR_INVALID_ARG; the GEMM routes are ETD_ERR_UNSUPPORTED for batches. With
 * opt->bc = ETD_BC_PERIODIC every problem is periodic (fields [N_y][N_x]) and flog may be nonzero;
 * Dirichlet batches take flog = 0.
 */
typedef struct etd_batch_s* etd_batch;
etd_status etd_batch_create(etd_batch* out, int count, const int64_t* N, const double* h, const double* D,
                            double tau, etd_scheme scheme, const etd_options* opt);

/* Advance every problem by nsteps >= 0 steps: u is a HOST array of `count` DEVICE pointers, u[i] the
 * dense field of problem i (shape [N[2i+1]-1][N[2i]-1], periodic [N[2i+1]][N[2i]], updated in place). Asynchronous on stream;
 * the pointer array itself may be reused as soon as the call returns. */
etd_status etd_batch_run(etd_batch b, void* const* u, int64_t nsteps, void* stream);

/* Total unknowns, launches per time step, and the tuned pencil pairs per tile of the first
 * max_groups step launches (any pointer may be NULL). */
etd_status etd_batch_info(etd_batch b, int64_t* unknowns, int* launches_per_step, int* tile_pairs, int max_groups);

/* The steady-state schedule chosen at creation: *parallel = 1 for parallel graph branches per pass,
 * 0 for the serial stream; *us_serial and *us_parallel = the creation-time trial's microseconds per
 * time step of each (0 where no trial ran: a single launch per pass, ETD_AUTOTUNE=0, or a forced
 * schedule). Any pointer may be NULL. */
etd_status etd_batch_schedule(etd_batch b, int* parallel, double* us_serial, double* us_parallel);

/* Release a batch. NULL is accepted. */
etd_status etd_batch_destroy(etd_batch b);

/* Static description of a status code. */
const char* etd_status_string(etd_status s);

/* Detail of the calling thread's most recent failure ("" if none). */
const char* etd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ETD_GB300_H */
