/*
 * smc.h -- C ABI of the GB300 (sm_103a) SMC hot path.
 *
 * The library evaluates the right-hand side of the multicomponent reacting
 * compressible Navier-Stokes equations (Emmett, Zhang & Bell, arXiv
 * 1309.7327, Sec. 2.1, eq. cns) on 3-D boxes of a structured grid with the
 * paper's 8th-order spatial discretisation (Sec. 2.2), and advances it with
 * spectral deferred corrections (Sec. 3.1, eq. expsdc) or multirate SDC
 * (Sec. 3.2): mode 1 (eq. mrupdate, explicit reactions on the fine nodes) or
 * mode 2 (eq. mrupdate2, reactions integrated implicitly on the coarse
 * nodes).  One GPU, one CUDA stream per handle.
 *
 * Units are CGS throughout (cm, g, s, K, erg); activation energies are in
 * cal/mol.  All functions return an smc_status and never abort.
 *
 * Array layout ("box layout").  A field set of C components over the cells
 * of all boxes is one contiguous array of doubles
 *     a[c * ncells + offset(b) + (k * ny_b + j) * nx_b + i]
 * component-major, boxes concatenated in grid order, each box [z][y][x]
 * with x fastest, interior cells only (no ghost cells).  ncells is the sum
 * of the boxes' cell counts.
 *
 * Conserved state U (NV = 5 + nspecies components, eq. cns):
 *     rho, rho*u, rho*v, rho*w, rho*E, rho*Y_1 .. rho*Y_ns
 * Primitive input of smc_prim_to_cons (NV components):
 *     u, v, w, T, p, Y_1 .. Y_ns
 *
 * Pointers.  U, dUdt and prim may be device pointers (cudaMalloc'd, or a
 * PyTorch CUDA tensor's data) or host pointers.  Device pointers are used in
 * place and the call is asynchronous on the handle's stream.  Host pointers
 * are staged through handle-owned device buffers and the call returns after
 * the result is back in host memory.  The caller owns U, dUdt and prim; the
 * handle owns everything else.
 *
 * Errors.  Argument errors are returned at once.  Conditions detected on the
 * device (Newton non-convergence of the temperature, T <= 0 or rho <= 0,
 * non-finite input) are recorded in a device status word and returned by the
 * next synchronising call (smc_synchronize, or any call given host
 * pointers).  smc_last_error gives a message for the last failure.
 *
 * Thread safety: a handle may be used by one host thread at a time.
 */
#ifndef SMC_H
#define SMC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smc_handle smc_handle;

typedef enum {
  SMC_OK = 0,
  SMC_ERR_ARG = 1,           /* invalid argument or unsupported configuration */
  SMC_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  SMC_ERR_OOM = 3,           /* device allocation failed */
  SMC_ERR_NONCONVERGED = 4,  /* temperature Newton iteration did not converge */
  SMC_ERR_NONPHYSICAL = 5,   /* rho <= 0, T <= 0 or a non-finite value */
  SMC_ERR_TIMEOUT = 6,       /* reserved: a bounded device wait gave up */
  SMC_ERR_STATE = 7          /* call out of order (e.g. use after destroy) */
} smc_status;

/* Boxes of a BoxLib-style box array (Sec. 4).  Box b covers the global cells
 * lo[3b..3b+2] .. hi[3b..3b+2] (inclusive, order x, y, z).  Boxes must not
 * overlap, and every ghost cell (4 per side, Sec. 2.5) of every box must map,
 * through the periodic wrap of the domain, onto a cell of some box. */
typedef struct {
  int nboxes;
  const int *lo, *hi;        /* [3 * nboxes] */
  int domain[3];             /* global cells in x, y, z */
  double dx[3];              /* cell size in x, y, z (cm) */
} smc_grid;

/* A reversible mass-action mechanism and its mixture transport model.
 * Thermodynamics: NASA 7-coefficient polynomials, one temperature range,
 *   cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4,
 *   h/RT = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T,
 *   s/R  = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7.
 * Rates (rho*omega_k of eq. NS:rY): k_f = A T^b exp(-Ea / (R_c T)),
 *   K_c = exp(-sum_k nu_k g_k/(R T)) (p_atm/(R_u T))^(sum_k nu_k),
 *   k_r = k_f / K_c, q = k_f prod c^nu' - k_r prod c^nu''.
 * Transport (the paper uses EGLIB; this library uses the model below):
 *   eta = eta_ref (T/T_ref)^eta_exp, lambda = cp eta / Pr,
 *   rho D_k = lambda / (cp Le_k), bulk viscosity xi = xi_ratio * eta.
 * Limits checked by smc_create (SMC_ERR_ARG otherwise): every reaction
 * conserves mass (sum_k nu_k W_k = 0 to 1e-9), has at most 4 species and 3
 * molecules per side; cp > 0 and the species' g/RT spread over less than
 * 400 on 200..3500 K (the FP64 range of the rate evaluation).
 * All arrays are host memory, copied by smc_create. */
typedef struct {
  int nspecies;              /* 1 .. 64 */
  int nreactions;            /* 0 .. 1024 */
  const double *W;           /* [ns] molecular weights, g/mol */
  const double *nasa7;       /* [ns * 7] a1..a7 per species */
  const int *nu_f;           /* [nr * ns] reactant coefficients (>= 0) */
  const int *nu_r;           /* [nr * ns] product coefficients (>= 0) */
  const double *A;           /* [nr] pre-exponential factors (mol, cm, s) */
  const double *b;           /* [nr] temperature exponents */
  const double *Ea;          /* [nr] activation energies, cal/mol */
  const double *Le;          /* [ns] Lewis numbers */
  double eta_ref, T_ref, eta_exp, Pr;
} smc_mechanism;

enum { SMC_BC_PERIODIC = 0, SMC_BC_OUTFLOW = 1 };
/* Boundary kind of each domain face.  y and z must be periodic.  x is
 * periodic, or SMC_BC_OUTFLOW on both ends: every x derivative in the four
 * cells next to an end then uses the boundary-lowered stencils of Sec. 2.2
 * (6th-, 4th- and 2nd-order centred diffusion and first derivatives at the
 * fourth, third and second cells, completely biased ones at the end cell),
 * without a characteristic boundary correction.  Outflow x needs at least
 * 8 cells along x and boxes at least 3 cells wide.  Other combinations
 * return SMC_ERR_ARG.  A NULL bc means periodic everywhere. */
typedef struct { int lo[3], hi[3]; } smc_bc;

/* Options for smc_set_option (value given as a double). */
enum {
  SMC_OPT_PRECISION = 0,       /* 0: FP64 everywhere (default); 1: mixed -- FP32 stencil, flux
                                  and transport arithmetic on float pairs, FP64 temperature,
                                  Gibbs energies, exponentials, rates and all accumulation */
  SMC_OPT_M47 = 1,             /* free parameters of the 8th-order narrow */
  SMC_OPT_M48 = 2,             /* stencil (Sec. 2.2); default 3557/44100, -2083/117600 */
  SMC_OPT_DIFFUSION_MODE = 3,  /* 0: correction velocity (default, Sec. 2.4); 1: reference species */
  SMC_OPT_REF_SPECIES = 4,     /* reference species index (default: last) */
  SMC_OPT_XI_RATIO = 5,        /* bulk viscosity xi = value * eta (default 0) */
  SMC_OPT_NEWTON_TOL = 6,      /* |dT| <= tol * T ends the iteration (default 1e-13) */
  SMC_OPT_NEWTON_MAXIT = 7,    /* at most this many Newton steps (default 50) */
  SMC_OPT_T_GUESS = 8,         /* Newton first guess in K (default 1000) */
  SMC_OPT_REACTIONS = 9,       /* 1: include rho*omega_k (default); 0: omit */
  SMC_OPT_SEGMENT = 10,        /* cells per thread along a stencil line (default 16) */
  SMC_OPT_PROFILE = 11,        /* 1: time every kernel launch with CUDA events (default 0) */
  SMC_OPT_USE_GRAPHS = 12,     /* 1 (default): replay recycled steps as one CUDA graph when the
                                  handle has a non-default stream and profiling is off; 0: launch
                                  kernels one by one */
  SMC_OPT_X_LAYOUT = 13,       /* x-direction lines of the current precision: 0 (default) read
                                  the box layout, 1 read an x-slowest copy made once per
                                  evaluation (nQ + 9 more ghosted planes of device memory) */
  SMC_OPT_MARCH = 14,          /* stencil-line kernel of the current precision.  FP64: 0 (default)
                                  evaluates every face from its 8-point window; 1, 2, 3 slide
                                  9-cell register windows along the line, one load per field
                                  and cell, in chunks of 16 / 32 / 8 cells (3 also keeps the
                                  pressure products of every face in shared memory for the
                                  species terms, at 2 resident blocks per SM).  Mixed: 1, 2, 3
                                  slide windows in chunks of 16 / 32 / 8 cells (3 keeps the
                                  pressure products of both faces of every cell in shared
                                  memory, at 2 resident blocks per SM; 0 is taken as 1;
                                  default 1) */
  SMC_OPT_RATES = 15,          /* production rates under SMC_OPT_PRECISION = 1: 0 (default)
                                  FP64 like the FP64 path; 1 FP32 mantissas after FP64 Gibbs
                                  energies, reaction exponents and exponent reductions
                                  (about 1e-6 relative; ignored in FP64 precision) */
  SMC_OPT_FINE_REPEAT = 16,    /* multirate fine nodes (Sec. 3.2): each coarse interval holds
                                  this many consecutive groups of reaction_substeps
                                  Gauss-Lobatto nodes; 1 (default) is type (b), more is
                                  type (c) (1..8; at most 64 fine intervals per step) */
  SMC_OPT_SDC_EXIT = 17,       /* eps >= 0; 0 (default) runs every sweep.  eps > 0: after each
                                  sweep compute the residual R^k = U_0 + dt q.F^k - U_M^k of
                                  eq. residual (for MRSDC the coarse and fine quadratures of
                                  f1 and f2) and end the step once |R^(k-1)| / |R^k| < 1 + eps
                                  or |R^k| = 0.  Reads the residual to the host every sweep
                                  (a stream synchronisation); steps are then launched one
                                  kernel at a time, not replayed as a graph */
  SMC_OPT_CHAIN_BLOCKS = 18,   /* cap on the resident blocks per SM of the multirate reaction
                                  chain, 0 (default) = the hardware limit; 1..16 reserve
                                  unused shared memory to enforce it (fewer resident threads,
                                  more L1 per thread for the chain's local arrays) */
  SMC_OPT_MR_MODE = 19,        /* multirate mode of smc_sdc_step with reaction_substeps >= 2:
                                  1 (default) explicit reactions on the fine nodes (eq.
                                  mrupdate); 2 reactions on the coarse nodes, integrated
                                  implicitly over each coarse interval by the BDF method,
                                  advection-diffusion on the fine nodes (eq. mrupdate2;
                                  at most 32 species) */
  SMC_OPT_BDF_RTOL = 20,       /* relative tolerance of the implicit reaction integration,
                                  0 < rtol < 1, default 1e-8 */
  SMC_OPT_BDF_ATOL = 21,       /* absolute tolerance of the implicit reaction integration in
                                  mass-fraction units (the weight of rho Y_k is
                                  atol rho + rtol |rho Y_k|), >= 0, default 1e-12 */
  SMC_OPT_PERSISTENT = 22,     /* launch shape of the multirate reaction chain and the
                                  sliding-window line kernels: 0 (default) one thread per cell
                                  or line segment, as many blocks as that takes; 1 one grid of
                                  the device's resident capacity (blocks per SM from the
                                  occupancy calculator x SM count) whose threads loop over the
                                  work items, so no partly filled last wave of blocks */
  SMC_OPT_ALU = 23             /* FP64 rate arithmetic moved to the integer and FP32 pipes
                                  (the FP64 pipe is the scarce one): 0 none; 1 (default) the
                                  exponentials of the production rates, the transport power law
                                  and the implicit integrator (smc_exp variant 1; within 2 ulp
                                  like variant 0); 2 also the products of the rate terms and of
                                  the temperature solve (smc_dmul: correctly rounded, the FP64
                                  unit's results bit for bit, but slower: the 64-bit integer
                                  multiplies cost more issue slots than they free) */
};

/* Kernel classes counted in smc_stats (launches always; times only while
 * SMC_OPT_PROFILE is 1, summed over the handle's lifetime). */
enum {
  SMC_K_PRIM = 0,       /* primitives, transport, ghost-cell gather */
  SMC_K_GRAD = 1,       /* velocity gradients for the mixed viscous terms */
  SMC_K_MARCH = 2,      /* narrow stencils + convective D, one direction */
  SMC_K_FINAL = 3,      /* correction-velocity terms and production rates */
  SMC_K_UPDATE = 4,     /* SDC node update */
  SMC_K_FINE = 5,       /* multirate fine-node reaction chain */
  SMC_K_CHEM = 6,       /* reaction-only evaluation */
  SMC_K_OTHER = 7,      /* primitive-to-conserved conversion, layout copies */
  SMC_K_BDF = 8,        /* implicit reaction integration (MRSDC mode 2) */
  SMC_NKERNELS = 9
};

typedef struct {
  long long n_rhs;           /* advection-diffusion(-reaction) RHS evaluations */
  long long n_react;         /* reaction-only evaluations (multirate fine nodes) */
  long long n_steps;         /* smc_sdc_step calls completed */
  unsigned int device_flags; /* last device status word read */
  int nvars;                 /* NV = 5 + nspecies */
  long long ncells;          /* interior cells over all boxes */
  long long device_bytes;    /* device memory held by the handle */
  long long launches[SMC_NKERNELS];   /* kernel launches per class */
  double kernel_ms[SMC_NKERNELS];     /* summed device time per class (profiling on) */
  int sweeps_done;           /* sweeps of the last smc_sdc_step */
  double residual[64];       /* |R^k| after sweep k of the last step (SMC_OPT_SDC_EXIT > 0
                                only; 0 otherwise): max over components of
                                max|R_c| / max|U_0,c| */
  /* implicit reaction integration (SMC_OPT_MR_MODE 2, smc_react_integrate),
     summed over every cell and call since the handle was created */
  long long bdf_steps;       /* accepted BDF steps */
  long long bdf_rejected;    /* steps rejected by the local error test */
  long long bdf_newton_failures;   /* attempts whose Newton iteration failed */
  long long bdf_evals;       /* production-rate evaluations */
  long long bdf_max_steps;   /* most accepted steps of one cell in one call */
  int schedule[4];           /* the schedule in use for the current precision: segment
                                length, x-line layout, line kernel (SMC_OPT_SEGMENT,
                                SMC_OPT_X_LAYOUT, SMC_OPT_MARCH) and launch shape
                                (SMC_OPT_PERSISTENT) */
} smc_stats;

/* Create a handle: validates the mechanism (limits above) and the grid,
 * uploads constants and builds the ghost-cell gather maps.  *out receives
 * the handle.  The current CUDA device is used.  On failure *out may still
 * receive a handle that holds the error message (smc_last_error); pass it
 * to smc_destroy. */
smc_status smc_create(const smc_grid *grid, const smc_mechanism *mech,
                      const smc_bc *bc, smc_handle **out);

/* Free the handle and everything it owns.  Accepts NULL. */
smc_status smc_destroy(smc_handle *h);

/* dUdt = full right-hand side of eq. cns at U (box layout, NV components):
 * primitives and transport, -D of the convective fluxes (8th-order centred
 * D), narrow-stencil (eqs. DaDu, H) viscous, conductive and diffusive terms,
 * the correction-velocity or reference-species closure (Sec. 2.4), and the
 * production rates.  Ghost cells are filled from U by periodic wrap. */
smc_status smc_rhs(smc_handle *h, const double *U, double *dUdt);

/* Advance U in place by one time step dt (s).
 *   reaction_substeps <= 1: single-rate SDC, eq. expsdc, with `nodes`
 *     Gauss-Lobatto nodes (3 or 5) and `sweeps` (>= 1) sweeps from the spread
 *     initial guess; f(U_0) is recycled from the previous step when U is the
 *     array the previous call left (call smc_invalidate after changing U).
 *   reaction_substeps = Y >= 2: multirate SDC, `nodes` coarse Gauss-Lobatto
 *     nodes and Y Gauss-Lobatto fine nodes in every coarse interval (type (b),
 *     Sec. 3.2; type (c) with SMC_OPT_FINE_REPEAT), Y <= 9.  Mode 1
 *     (SMC_OPT_MR_MODE, default; eq. mrupdate): advection-diffusion on the
 *     coarse nodes, explicit reactions on the fine nodes.  Mode 2 (eq.
 *     mrupdate2): reactions on the coarse nodes, integrated implicitly over
 *     every coarse interval (as smc_react_integrate, with the forcing of the
 *     sweep's other terms), advection-diffusion on the fine nodes with
 *     forward-Euler substeps; at most 10 fine intervals per coarse interval
 *     and 32 species. */
smc_status smc_sdc_step(smc_handle *h, double *U, double dt, int nodes,
                        int sweeps, int reaction_substeps);

/* U from primitive fields (u, v, w, T, p, Y_k): rho from the ideal-gas law,
 * rho E = rho (sum_k Y_k e_k(T) + |u|^2/2).  Same layout rules as U. */
smc_status smc_prim_to_cons(smc_handle *h, const double *prim, double *U);

/* Set the CUDA stream (a cudaStream_t) used by later calls; NULL = default. */
smc_status smc_set_stream(smc_handle *h, void *stream);

/* Set an SMC_OPT_* option; invalidates the recycled f(U_0). */
smc_status smc_set_option(smc_handle *h, int key, double value);

/* Counters and sizes. */
smc_status smc_get_stats(smc_handle *h, smc_stats *out);

/* Wait for the handle's stream, then return (and clear) any device-detected
 * error. */
smc_status smc_synchronize(smc_handle *h);

/* Drop the cached f(U_0) of the last step. */
smc_status smc_invalidate(smc_handle *h);

/* Autotune the stencil kernels for the handle's current precision: time
 * one right-hand-side evaluation at U (device memory, box layout) for every
 * segment length (cells per thread along a stencil line: 8, 16, 32, 64),
 * both layouts of the x-direction lines (0: read the box layout directly;
 * 1: read a copy with x the slowest index, made once per evaluation) and
 * every stencil-line kernel of the precision (SMC_OPT_MARCH), then the
 * winner with the other launch shape (SMC_OPT_PERSISTENT), and keep the
 * fastest.  *segment, *x_layout and *march (each may be NULL) receive the
 * choice.  Synchronises the handle's stream. */
smc_status smc_autotune(smc_handle *h, const double *U, int *segment, int *x_layout, int *march);

/* Collocation data used by smc_sdc_step (host computation, no GPU needed).
 * smc_collocation: the `nodes` Gauss-Lobatto nodes on [0, 1] (tau[nodes])
 * and the node-to-node integration matrix S[(nodes-1) * nodes] of Sec. 3.1,
 * s_mj = integral over [tau_m, tau_{m+1}] of the Lagrange polynomial L_j.
 * smc_multirate_collocation: coarse nodes t1[coarse] and fine nodes
 * t2[M2 + 1] of Sec. 3.2 -- `repeat` consecutive groups of `fine`
 * Gauss-Lobatto nodes in every coarse interval (type (b) for repeat = 1,
 * type (c) otherwise), M2 = (coarse-1)(fine-1) repeat -- and the matrices
 * S21[M2 * coarse] (coarse Lagrange basis) and S22[M2 * (M2 + 1)] (the
 * piecewise basis of each group) of eq. mrupdate, per unit time step.  All
 * arrays are caller-owned host memory. */
smc_status smc_collocation(int nodes, double *tau, double *S);
smc_status smc_multirate_collocation(int coarse, int fine, int repeat, double *t1, double *t2,
                                     double *S21, double *S22);

/* The FP64 right-hand side of smc_rhs for ONE triply periodic box of
 * n[0] x n[1] x n[2] cells (spacing dx, cm) without any device allocation.
 * The paper has no counterpart.  It exists for callers that cannot call
 * cudaMalloc: applications whose framework owns all device memory in a fixed
 * arena, and loops that must not pay the implicit synchronisation of
 * cudaMalloc/cudaFree.
 * U and dUdt are caller-owned arrays in the box layout, device memory of the
 * current device (SMC_ERR_ARG otherwise: there is no host staging); mech is
 * host memory.  Default options (correction-velocity mode, default stencil
 * parameters, reactions on).  All scratch, tables and constants live in one
 * static device array of 20 MiB that every GPU loading the library reserves
 * until the process exits; a box whose scratch would not fit (about 16^3
 * cells with 21 species, 24^3 with 3), or with a side above 65536, returns
 * SMC_ERR_ARG.  The first call on a device looks up that array's address
 * (cudaGetSymbolAddress).  Tables are copied from host memory with
 * cudaMemcpyAsync on `stream` (a cudaStream_t, NULL = default) and the call
 * waits for the stream and returns the device status of the evaluation, so
 * it cannot be issued while `stream` is being captured into a CUDA graph.
 * Calls share the array and it keeps the last call's contents: calls that
 * overlap on the GPU race and must be serialised by the caller. */
smc_status smc_rhs_noalloc(const int n[3], const double dx[3], const smc_mechanism *mech,
                           const double *U, double *dUdt, void *stream);

/* The appendix heat-equation problems (App. A, T1/T2):
 *   u_t = (a u_x)_x + (b u_y)_y + exp(-t) G(x, y)
 * on a periodic N x N grid of spacing h (N >= 8), both terms by the narrow
 * stencil of Sec. 2.2 with free parameters m47, m48, advanced by nsteps
 * SDC steps (Sec. 3.1: `nodes` Gauss-Lobatto nodes, `sweeps` sweeps) of dt
 * from t0.  a, b, G (may be NULL: no source) and u are caller-owned device
 * arrays of N*N doubles, row-major with x fastest; u is advanced in place.
 * The step recycles f(U_M) as the next f(U_0).  *n_evals (may be NULL)
 * receives the number of operator evaluations.  Allocates its scratch
 * ((2 + 2 (nodes - 1)) N^2 doubles) and synchronises `stream` (a
 * cudaStream_t, NULL = default) before returning.  SMC_ERR_ARG for bad
 * sizes or host pointers, SMC_ERR_OOM, SMC_ERR_CUDA. */
smc_status smc_heat2d(int N, double h, const double *a, const double *b, const double *G,
                      double m47, double m48, double t0, double dt, int nsteps, int nodes,
                      int sweeps, double *u, long long *n_evals, void *stream);

/* The exponentials used by the production rates (table-driven methods, not
 * the paper's: Sec. 2.1 only needs exp), applied elementwise y[i] = exp(x[i])
 * on the device for accuracy tests.  variant 0: the table method in FP64
 * arithmetic; variant 1: the same decomposition with the argument reduction
 * in 128-bit fixed point, exp(r) as a float pair and the result assembled in
 * 64-bit fixed point (integer and FP32 pipes; SMC_OPT_ALU).  x and y are
 * caller-owned device arrays of n doubles (n >= 0).  Arguments with
 * |x| >= 512 are clamped to [-708, 709].  Synchronous; returns SMC_ERR_ARG
 * for null arrays, host pointers or another variant, SMC_ERR_CUDA if the
 * launch fails. */
smc_status smc_exp(const double *x, double *y, long long n, int variant);

/* y[i] = a[i] * b[i] by the integer-pipe product the production rates use
 * under SMC_OPT_ALU = 2 (the 106-bit product of the significands, rounded to
 * nearest even), for its exactness test against the FP64 product.  Device
 * arrays of n doubles; synchronous; SMC_ERR_ARG for null or host arrays,
 * SMC_ERR_CUDA if the launch fails. */
smc_status smc_dmul(const double *a, const double *b, double *y, long long n);

/* Implicit integration of the reactions alone, cell by cell (the coarse
 * reaction term of MRSDC mode 2, eq. mrupdate2):
 *   dU/dtau = R(U) + G,  U(0) = U,  0 <= tau <= dt,
 * R the production rates of the species components (no other component
 * has a reaction source), G a constant forcing (NULL: zero).  The
 * non-species components move linearly; the species are integrated by a
 * variable-order (1..5), variable-step BDF method with a Newton iteration on
 * the analytic Jacobian at fixed density and internal energy, error
 * weights SMC_OPT_BDF_ATOL rho + SMC_OPT_BDF_RTOL |rho Y_k|.  U, G and
 * Uout are caller-owned device arrays in the box layout (NV components);
 * Uout receives U(dt) and may be U itself.  At most 32 species.
 * Stream-ordered on the handle's stream; a cell whose temperature solve
 * fails or whose step size collapses sets the device status reported by
 * the next synchronising call (SMC_ERR_NONCONVERGED).  SMC_ERR_ARG for bad
 * arguments or host pointers. */
smc_status smc_react_integrate(smc_handle *h, const double *U, const double *G, double dt,
                               double *Uout);

/* Measured throughput of one fused multiply-add pipe of the current device:
 * the denominator of the arithmetic rooflines (Sec. 2.3 counts the flops of
 * the stencils; this measures the rate they can run at on this GPU).
 *   kind 0: FP64 FMA (DFMA); 1: FP32 FMA; 2: paired FP32 FMA (two per lane
 *   and instruction); 3: FP64 FMA on one active lane per warp (flops of the
 *   active lanes: what scalar FP64 work costs in warp-cooperative code).
 * One untimed launch, then one launch of multiProcessorCount x 4 blocks of
 * 256 threads, each thread running 8 independent FMA chains for `iters`
 * iterations, timed with CUDA events on a private stream.  *flops_per_s
 * receives 2 x FMAs / s (required), *ms the timed launch's duration and
 * *sm_count the device's SM count (both may be NULL).  Allocates and frees
 * one small device buffer and synchronises.  SMC_ERR_ARG for kind outside
 * 0..3 or iters outside 1..2^40, SMC_ERR_OOM, SMC_ERR_CUDA. */
smc_status smc_fma_throughput(int kind, long long iters, double *flops_per_s, double *ms,
                              int *sm_count);

/* Message describing the last error on this handle ("" if none).  The
 * string is owned by the handle. */
const char *smc_last_error(smc_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* SMC_H */
