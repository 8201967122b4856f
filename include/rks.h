/*
 * rks.h -- C ABI of the batched closed-shell Kohn-Sham (B3LYP/STO-3G) SCF
 * engine for one GB300 (sm_103a).
 *
 * What it computes (arXiv 2311.01135, Section 3.1, Eq. 1): for each molecule
 * (atomic numbers Z, positions R) the self-consistent solution of
 *     [V + T + J(rho) + K(rho) + V_xc(rho)] C = S C eps,   rho = C D C^T,
 * D_ii = 2 for the N_el/2 lowest orbitals, with the Coulomb and exchange
 * contractions of the two-electron tensor I^2e written in Eq. 1, B3LYP
 * exchange-correlation (Section 3.2, "Libxc") in the STO-3G basis
 * (Section 3.3), and the HL gap of Section 3.1 (reported here as
 * eps_LUMO - eps_HOMO > 0).  Outputs match the labels of the paper's dataset
 * (Section 4: energy, HOMO, LUMO).
 *
 * Conventions shared by every call:
 *  - Return value 0 (RKS_OK) on success, a negative RKS_E* code otherwise;
 *    rks_strerror() names it.  Numerical outcomes of one molecule (not
 *    converged, non-finite, ill-conditioned S) are reported in
 *    rks_result_t.status, not as call errors.
 *  - Every input array is read during the call and copied; the library never
 *    keeps a caller pointer.  Every output buffer is caller-owned.
 *  - Coordinates are bohr unless rks_options.coords_in_angstrom is set
 *    (1 bohr = 0.52917721092 Angstrom).  Energies are Hartree.
 *  - AO order: atoms in input order; per heavy atom (C, N, O, F) 1s, 2s, 2px,
 *    2py, 2pz; per H 1s.  Matrices are nbf x nbf, row-major, FP64.
 *  - Supported elements: H, C, N, O, F.  The electron count must be even.
 *  - A context owns one CUDA device, its streams and all device memory.  It
 *    is safe to call rks_submit / rks_poll / rks_wait / rks_result from
 *    several host threads.
 */
#ifndef RKS_H
#define RKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define RKS_OK 0
#define RKS_EINVAL (-1)    /* bad argument: element, natom, odd N_el, non-finite xyz, nbf too large */
#define RKS_ENOMEM (-2)    /* device or host allocation failed, or request exceeds the HBM budget */
#define RKS_EAGAIN (-3)    /* submission queue full; retry later */
#define RKS_ENOTREADY (-4) /* ticket not finished yet */
#define RKS_ECUDA (-5)     /* a CUDA call failed (message via rks_last_error) */
#define RKS_ETIMEOUT (-6)  /* rks_wait timed out */
#define RKS_ENOTFOUND (-7) /* unknown or already released ticket */
#define RKS_EDEVICE (-8)   /* a device-side bounded wait or bounds check gave up */

/* ---------------------------------------------------- per-molecule status */
#define RKS_STATUS_OK 0
#define RKS_STATUS_NOT_CONVERGED 1 /* "converge" protocol hit max_iters */
#define RKS_STATUS_NONFINITE 2     /* a NaN/Inf appeared in F, E or eps */
#define RKS_STATUS_S_ILL 3         /* min eig(S) < 1e-8 */
#define RKS_STATUS_EIGH 4          /* Jacobi did not reach tolerance */

/* ---------------------------------------------------------- ticket state */
#define RKS_PENDING 0
#define RKS_RUNNING 1
#define RKS_DONE 2
#define RKS_FAILED 3

/* --------------------------------------------------------------- precision */
#define RKS_FP64 0  /* every step in FP64 */
#define RKS_MIXED 1 /* FP32 ERIs / J/K / grid + FP64 linear algebra and energy, FP64 final correction */

#define RKS_MAX_NBF 224 /* largest basis a molecule may have (20-30 heavy atoms reach ~200); above
                           96 functions a molecule takes the global-memory J/K, grid and SCF kernels */

/* ---------------------------------------------------------- initial guess */
#define RKS_GUESS_SAD 0  /* superposed neutral atoms: 1s/2s space full, 2p^(Z-4) spherically averaged */
#define RKS_GUESS_CORE 1 /* diagonalise the core Hamiltonian T + V */

typedef struct rks_ctx rks_ctx;
typedef struct rks_batch rks_batch;

typedef struct rks_options {
    int32_t basis;          /* 0 = STO-3G (only value) */
    int32_t n_rad;          /* radial points per atom (Treutler-Ahlrichs M4), default 50 */
    int32_t n_theta;        /* Gauss-Legendre nodes in cos(theta), default 12 */
    int32_t n_phi;          /* uniform azimuthal points, default 24 */
    int32_t becke_iters;    /* Becke smoothing iterations, default 3 */
    int32_t precision;      /* RKS_FP64 or RKS_MIXED */
    int32_t fixed_iters;    /* > 0: run exactly this many SCF iterations, then the final step;
                               0: iterate to convergence (e_tol, err_tol), at most max_iters */
    int32_t max_iters;      /* cap for the converge protocol, default 100 */
    double e_tol;           /* |E_k - E_(k-1)| threshold (Ha), default 1e-9 */
    double err_tol;         /* max |X^T(FDS - SDF)X| threshold, default 1e-6 */
    int32_t diis_space;     /* DIIS history length (1..8), default 8 */
    int32_t coords_in_angstrom;
    int32_t xc;             /* 1 = B3LYP (default); 0 = Hartree-Fock test mode (a0 = 1, no V_xc) */
    int32_t max_slots;      /* serving: most molecules in one cohort, default 4096 */
    uint64_t hbm_budget_bytes; /* serving: cap on the device memory of all cohorts in flight;
                                  0 = 85% of the memory free when the context is created */
    int32_t device;         /* CUDA device ordinal, default 0 */
    int32_t use_graphs;     /* capture fixed-iteration loops in CUDA graphs, default 1 */
    int32_t pad0;
    double fix_theta;       /* RKS_MIXED final step: quartets with Schwarz bound Q_pq Q_rs >= fix_theta
                               are recomputed in FP64 and replace their FP32 store values in J/K;
                               0 disables; default 0.1 */
    int32_t grid_tc;        /* RKS_MIXED: 1 = grid contractions on the tensor cores (tcgen05, 3xTF32)
                               for each molecule with nbf <= 80 and <= 60 shells, decided per
                               molecule (default); the others, and every molecule when 0, take
                               the CUDA-core grid kernel */
    int32_t guess;          /* initial density: RKS_GUESS_SAD (default) or RKS_GUESS_CORE */
    int32_t max_cohorts;    /* serving: most batches ("cohorts") in flight at once, each on its own
                               stream, default 4 */
    int32_t admit_wait_us;  /* serving: while other cohorts run, a partial cohort (fewer than
                               max_slots molecules) is admitted once its oldest request has waited
                               this long (microseconds), default 20000 */
    int32_t grid_chunks;    /* thread blocks per molecule of the grid kernels (0 = default: 16 on the
                               mixed path; on the FP64 path 16, or more for batches too small to
                               fill the GPU); changes the grouping of the V_xc sums, so mixed
                               results move at ~1e-7 */
    int32_t jk_chunks;      /* thread blocks per molecule of the J/K kernel (0 = default: 8, or more
                               for batches too small to fill the GPU); results are bit-identical
                               for any value on the mixed path */
    int32_t iter_precision; /* RKS_MIXED: precision of the Fock builds inside the SCF iterations,
                               bit flags: RKS_ITER_JK_FINAL = J/K as in the final step (FP64
                               products and the FP64 recompute of the largest quartets),
                               RKS_ITER_GRID_FINAL = grid pass as in the final step (density
                               contraction on the CUDA cores); default 0 (both at iteration
                               precision) */
    int32_t direct_scf;     /* where J/K get the two-electron integrals (paper Section 5,
                               "Recomputation"): RKS_DIRECT_NEVER (default) computes the
                               Schwarz-screened packed store once and streams it every Fock
                               build; RKS_DIRECT_ALWAYS keeps no store and recomputes every kept
                               quartet inside each J/K pass (the mixed final step recomputes
                               them in FP64); RKS_DIRECT_AUTO does so only for a batch whose
                               packed stores would take more than 70% of the free device memory */
    double recheck_err;     /* RKS_MIXED, fixed protocol: a molecule whose DIIS error max|e|
                               after the fixed iterations exceeds recheck_err is run again from
                               the initial guess, the same number of iterations, with both Fock
                               builds at the final step's precision, before the final step;
                               0 disables.  A molecule's decision depends on it alone.
                               Default 1e-4 */
    double recheck_fp64_err; /* RKS_MIXED, fixed protocol: a molecule whose DIIS error after the
                               fixed iterations exceeds recheck_fp64_err, or whose status is not
                               OK, has not converged and is redone on the FP64 path (paper
                               Section 3.2, "Numerical Error": the float32 results stand for the
                               converged molecules, the rest are recomputed in float64); its
                               result is the FP64 path's.  The redo runs as a batch of its own
                               on its own stream, beside the precise reruns and the final step.
                               0 disables.  Default 3e-4 (above it, a precise rerun of the
                               9-11-heavy-atom workload missed the FP64 gap by 1.2e-4 Ha) */
} rks_options;

#define RKS_ITER_JK_FINAL 1
#define RKS_ITER_GRID_FINAL 2

#define RKS_DIRECT_NEVER 0
#define RKS_DIRECT_ALWAYS 1
#define RKS_DIRECT_AUTO 2

/* One molecule's outputs: the labels the paper's dataset records per
 * conformer (Section 4: energy, HOMO, LUMO, HL gap) and the SCF bookkeeping
 * of Section 3.1's iteration. */
typedef struct rks_result_t {
    int32_t status;   /* RKS_STATUS_* */
    int32_t nbf;      /* basis size N of Section 3.1 (STO-3G, Section 3.3) */
    int32_t n_occ;    /* doubly occupied orbitals, N_electrons/2 (the D_ii = 2 entries of Eq. 1) */
    int32_t iters;    /* SCF iterations run (Section 3.1's iteration i), excluding the final step */
    double e_total;   /* total energy (Ha) of the density that entered the last Fock build */
    double e_homo;    /* eps[n_occ - 1]: eps of Eq. 1, ascending */
    double e_lumo;    /* eps[n_occ] */
    double gap;       /* HL gap of Section 3.1, reported as e_lumo - e_homo > 0 */
    double e_xc;      /* exchange-correlation energy of the B3LYP V_XC of Eq. 1 (Section 3.2, "Libxc"),
                         without the exact-exchange part carried by K */
    double e_nuc;     /* nuclear repulsion */
    double latency_s; /* submit -> done (serving API); batch wall time per molecule (batch API) */
    int32_t paper_converged; /* the paper's convergence flag (Section 3.2, "Numerical Error",
                                footnote): std of the last 5 energies < 0.01, taken in Ha */
    int32_t rechecked;       /* 1: the molecule was run again at the final step's precision
                                (rks_options.recheck_err); 2: redone on the FP64 path
                                (rks_options.recheck_fp64_err) */
    double err_max;   /* max |X^T (F D S - S D F) X| of the last SCF iteration */
    double de_last;   /* |E_k - E_(k-1)| of the last SCF iteration */
} rks_result_t;

/* Fill *o with the defaults listed above. */
int rks_options_default(rks_options *o);

/* Number of STO-3G basis functions of a molecule (no context needed);
 * negative RKS_EINVAL for an unsupported element or natom <= 0. */
int rks_nbf(int32_t natom, const int32_t *Z);

/* Device bytes one molecule adds to a batch under `options` (NULL: the
 * defaults), no context or device needed: its packed two-electron store (the
 * unscreened capacity of Section 3.2's 8-fold-symmetric I^2e; none under
 * RKS_DIRECT_ALWAYS), grid, FP64 matrices, accumulators and state.  The
 * paper's memory limit per molecule (Section 5: N <= 70 within 940 MB of
 * on-chip memory) becomes here the admission figure the serving worker holds
 * against hbm_budget_bytes.  Z: natom atomic numbers (read only).  Returns the
 * byte count, or RKS_EINVAL for natom <= 0, a null Z, an unsupported element
 * or a basis above RKS_MAX_NBF. */
int64_t rks_mol_bytes(const rks_options *options, int32_t natom, const int32_t *Z);

/* The tensor-core grid kernel's column plan of a molecule (no context
 * needed; mixed path, Section 3.1 V_xc on the grid).  The kernel's threads own
 * AO columns in four quarters of NQ = 4, 8, 12, 16 or 20 (padded basis 4 NQ);
 * a quarter is NQ / 5 units of five columns (a heavy atom's 1s, 2s, 2px, 2py,
 * 2pz, or up to five hydrogens) and NQ % 5 single hydrogen columns.
 * plan: caller-owned, RKS_TC_PLAN_INTS int32 written:
 *   [q * 5 + k], k < NQ / 5: unit word of quarter q: bit 31 set for a heavy
 *       atom; atom indices (0-based, molecule order) in 6-bit fields, field r
 *       for slot r, 63 = empty slot (a heavy unit uses field 0 only)
 *   [q * 5 + 4]: atom indices of the quarter's single columns, same fields
 *   [20 + c], c < 80: AO index of the kernel's column c (-1: padding)
 * Returns NQ, 0 when the kernel does not take the molecule (more than 63
 * atoms, a basis above 80 functions, or more heavy atoms than units at every
 * NQ; the CUDA-core grid kernel runs it), or RKS_EINVAL for invalid input. */
#define RKS_TC_PLAN_INTS 100
int rks_tc_plan(int32_t natom, const int32_t *Z, int32_t *plan);

const char *rks_strerror(int code);
/* Last CUDA / internal error message of the context (or the library when ctx is NULL). */
const char *rks_last_error(rks_ctx *ctx);

/* ------------------------------------------------------------ context */
/* Create a context on options->device: allocates streams and the constant
 * tables (Boys function table of the integral code, Section 3.2 "Libcint";
 * radial and angular quadrature tables of the grid), starts the serving
 * worker thread.  options may be NULL (defaults); *out receives the context,
 * owned by the caller until rks_destroy.
 * Errors: RKS_EINVAL (bad options), RKS_ECUDA (no device), RKS_ENOMEM. */
int rks_create(const rks_options *options, rks_ctx **out);
/* Stops the worker (queued and in-flight tickets are failed), frees device memory. */
int rks_destroy(rks_ctx *ctx);
/* The context's compute stream (a cudaStream_t), for timing with events. */
void *rks_stream(rks_ctx *ctx);

/* ------------------------------------------------------- serving API */
/* Queue one molecule: the inputs of a DFT computation, atomic numbers and
 * positions (Section 3.1), to be run through the iteration of Eq. 1.
 * Non-blocking: copies Z[natom] and xyz[natom*3] (row-major) and returns a
 * ticket in *ticket_out.  Continuous batching: the worker thread
 * keeps up to max_cohorts batches in flight, each on its own CUDA stream, and
 * admits queued molecules as a new cohort whenever the HBM budget has room
 * (a full cohort at once, a partial one when the GPU is idle or the oldest
 * request has waited admit_wait_us).  It advances every cohort a few SCF
 * iterations at a time without blocking (CUDA events and an asynchronous
 * read of the count of molecules still iterating); converged molecules drop
 * out of the work at once, and a cohort retires, publishing its tickets and
 * returning its memory for back-fill, after its final step.  A molecule's
 * result does not depend on which cohort it ran in.
 * Errors: RKS_EINVAL (validation as above), RKS_EAGAIN (queue full). */
int rks_submit(rks_ctx *ctx, int32_t natom, const int32_t *Z, const double *xyz,
               uint64_t *ticket_out);
/* Queue nmol molecules at once (Z and xyz concatenated, natom[m] atoms each),
 * all-or-nothing: every molecule is validated before any is queued, and they
 * reach the worker together (one admission decision).  tickets_out[nmol].
 * Errors: RKS_EINVAL (first invalid molecule named by rks_last_error),
 * RKS_EAGAIN. */
int rks_submit_batch(rks_ctx *ctx, int32_t nmol, const int32_t *natom, const int32_t *Z,
                     const double *xyz, uint64_t *tickets_out);
/* Non-blocking state query of a ticket from rks_submit: *state_out gets
 * RKS_PENDING (queued), RKS_RUNNING (its cohort is in Section 3.1's
 * iterations), RKS_DONE or RKS_FAILED.  Errors: RKS_EINVAL, RKS_ENOTFOUND. */
int rks_poll(rks_ctx *ctx, uint64_t ticket, int32_t *state_out);
/* Block the calling host thread until the ticket is done or timeout_s passes. */
int rks_wait(rks_ctx *ctx, uint64_t ticket, double timeout_s);
/* Copy the result of a finished ticket and release it: the energy, the
 * orbital energies eps and the density rho = C D C^T of Eq. 1 (Section 3.1),
 * HOMO, LUMO and gap (the labels of Section 4).  eps_out (nbf values,
 * ascending) and D_out (nbf*nbf, the output total density) may be NULL;
 * cap_nbf is their capacity in basis functions (RKS_EINVAL if smaller than
 * nbf).  Errors: RKS_ENOTREADY, RKS_ENOTFOUND; for a failed ticket (released
 * by this call) RKS_ENOMEM when the molecule alone exceeds the HBM budget,
 * RKS_ECUDA otherwise. */
int rks_result(rks_ctx *ctx, uint64_t ticket, rks_result_t *out, double *eps_out,
               double *D_out, int32_t cap_nbf);

/* --------------------------------------------------------- batch API */
/* A batch is a fixed set of molecules resident on the device; used by the
 * benchmark (device-resident inputs) and the parity tests.  Z and xyz are the
 * concatenation of every molecule's atoms; natom[m] gives the split.
 * Setup copies the inputs to the device (host->device happens here).
 * Errors: RKS_EINVAL, RKS_ENOMEM, RKS_ECUDA. */
int rks_batch_create(rks_ctx *ctx, int32_t nmol, const int32_t *natom, const int32_t *Z,
                     const double *xyz, rks_batch **out);
/* Enqueue the whole method of Section 3.1 for every molecule of the batch
 * (iteration 0: integrals incl. I^2e under its 8-fold symmetry, Section 3.2
 * footnote, and the grid; then the SCF iterations and the final step) on the
 * context stream and return without waiting.  For the converge protocol the
 * call reads the count of molecules still iterating every 4 iterations and
 * stops when it reaches zero; with recheck_err set it reads the count of
 * molecules to run again once, after the fixed iterations. */
int rks_batch_run(rks_batch *b);
/* Wait for the batch's work to finish; RKS_EDEVICE if a kernel reported a
 * bounded-wait or bounds failure. */
int rks_batch_sync(rks_batch *b);
/* Results of molecule m (after sync), same buffers and fields as rks_result. */
int rks_batch_result(rks_batch *b, int32_t m, rks_result_t *out, double *eps_out, double *D_out,
                     int32_t cap_nbf);
/* Free the batch's device memory (waits for its work). */
int rks_batch_destroy(rks_batch *b);

/* ------------------------------------------------- stage-level entries */
/* Run only the iteration-0 steps of Section 3.1 (V, T, S, I^2e: one-electron
 * integrals, Schwarz screening, packing, ERIs; the grid; the orthogonaliser
 * and the initial density) for the batch. */
int rks_batch_setup(rks_batch *b);
/* With the batch set up, build the operator of Eq. 1 at the given densities
 * rho (one nbf*nbf FP64 matrix per molecule, concatenated): J(rho), K(rho),
 * V_XC(rho), E_xc and E at rho (read back with rks_batch_dump).
 * final_step = 1 uses the precision of the final correction, 0 the
 * iterations' precision (rks_options.iter_precision). */
int rks_batch_fock(rks_batch *b, const double *D_all, int32_t final_step);

/* Copy a per-molecule array out for inspection (parity tests).
 * what: see RKS_DUMP_*.  Returns the number of bytes written, or a negative
 * error (RKS_EINVAL if cap is too small). */
#define RKS_DUMP_PAIRS 0    /* kept shell pairs: int32 [npair][2] (P, Q in packing shell order) */
#define RKS_DUMP_PAIR_Q 1   /* Schwarz Q of the kept pairs: double [npair] */
#define RKS_DUMP_ROW_OFF 2  /* element offset of every kept pair's row: int64 [npair + 1] */
#define RKS_DUMP_STORE 3    /* packed ERI values: double [n] (FP32 stores are widened) */
#define RKS_DUMP_S 4        /* overlap, double [nbf*nbf] */
#define RKS_DUMP_T 5        /* kinetic */
#define RKS_DUMP_V 6        /* nuclear attraction */
#define RKS_DUMP_GRID 7     /* grid points: double [npts][4] (x, y, z, w), padding removed */
#define RKS_DUMP_J 8        /* last Coulomb matrix */
#define RKS_DUMP_K 9        /* last exchange matrix K_std (no -a0/2 factor) */
#define RKS_DUMP_VXC 10     /* last V_xc */
#define RKS_DUMP_D 11       /* current density (input of the last Fock build) */
#define RKS_DUMP_F 12       /* last Fock matrix */
#define RKS_DUMP_EPS 13     /* orbital energies [nbf] */
#define RKS_DUMP_X 14       /* S^-1/2 */
#define RKS_DUMP_SCALARS 15 /* double [10]: E, E_xc, E_nuc, n_pair_all, n_quartets, store elements, npts,
                               near-tie count, and the screened work of one tensor-core grid pass:
                               sum over 128-point blocks of 128 n_sig^2 (n_sig: AOs significant in
                               the block), iterations, final step (0 for molecules the tensor-core
                               kernel does not take) */
#define RKS_DUMP_QUARTETS 16 /* kept quartet count per row: int32 [npair] */
int64_t rks_batch_dump(rks_batch *b, int32_t m, int32_t what, void *out, int64_t cap_bytes);

/* ------------------------------------------------------ profiling */
typedef struct rks_stage_time {
    char name[24];
    int32_t launches; /* kernel launches recorded since the last reset */
    double ms;        /* summed CUDA-event time of those launches */
    double units;     /* algorithmic work processed (bytes or flops, per stage) */
} rks_stage_time;
/* Record CUDA events around every stage launch on the context stream (on = 1). */
int rks_profile_enable(rks_ctx *ctx, int32_t on);
/* Read and reset per-stage totals; returns the number of stages written. */
int rks_profile_read(rks_ctx *ctx, rks_stage_time *out, int32_t cap);

/* ------------------------------------------------------ unit entries */
/* Boys function F_m(T) for m = 0..mmax at n arguments, by the device kernel
 * (tabulated Taylor expansion + asymptotic form).  out is [n][mmax+1].
 * precision RKS_FP64 or RKS_MIXED (FP32).  Host buffers. */
int rks_eval_boys(rks_ctx *ctx, int32_t mmax, int32_t n, const double *T, double *out,
                  int32_t precision);
/* B3LYP energy density and potentials (e, v_rho, v_sigma) at n points of
 * (rho, sigma = |grad rho|^2), by the device kernel (the V_XC of Eq. 1,
 * Section 3.2 "Libxc").  Host buffers.  precision RKS_FP64 or RKS_MIXED
 * (FP32), anything else RKS_EINVAL.  Allocates and frees device memory per
 * call (see rks_eval_xc_noalloc for callers that cannot). */
int rks_eval_xc(rks_ctx *ctx, int32_t n, const double *rho, const double *sigma, double *e,
                double *v_rho, double *v_sigma, int32_t precision);

/* ------------------------------------------------------ measurement */
/* Peak rate of one operation on the context's device, measured by a probe
 * kernel (the roofline denominators of kernels bound by that operation; the
 * paper has no counterpart).  kind: RKS_PROBE_FP32_FMA or RKS_PROBE_FP64_FMA
 * (flop/s, 2 per FMA, every SM full of independent FMA chains), or
 * RKS_PROBE_TF32_MMA (flop/s of back-to-back dense tcgen05.mma kind::tf32,
 * M = 128, N = 256, K = 8, on every SM).  Best of three timed launches after
 * one warm-up, CUDA events on the context stream; synchronous, ~0.1 s.
 * Errors: RKS_EINVAL (kind, null), RKS_ECUDA, RKS_EDEVICE (a bounded wait gave up). */
#define RKS_PROBE_FP32_FMA 0
#define RKS_PROBE_FP64_FMA 1
#define RKS_PROBE_TF32_MMA 2
int rks_probe_peak(rks_ctx *ctx, int32_t kind, double *ops_per_s);

/* ------------------------------------------------------ diagnostics */
/* Exercise the device-side failure path without a fault: one block waits on
 * an mbarrier that nothing ever arrives at, polling at most `spins` times
 * (1 .. 2^24), the same bounded wait the tensor-core kernels use.  Returns
 * RKS_EDEVICE when the wait gave up (the expected outcome), after which the
 * context stays usable.  RKS_EINVAL for spins out of range. */
int rks_selftest_bounded_wait(rks_ctx *ctx, int32_t spins);

/* ------------------------------------------- allocation-free XC entry */
/* The paper has no counterpart: this is a deployment variant of rks_eval_xc.
 * Same arguments, same kernel, same results (bit-identical), but it allocates
 * nothing: inputs and outputs are staged through one static device array
 * of 5 * RKS_XC_NOALLOC_MAX doubles (2.5 MiB) that the library holds per
 * device, so no cudaMalloc / cudaFree runs.  It is for callers that cannot
 * allocate device memory (a process whose memory is promised to the serving
 * budget) or cannot afford cudaFree's wait for the whole device (cohorts in
 * flight on other streams).
 *  - n must be 1 .. RKS_XC_NOALLOC_MAX; larger n returns RKS_EINVAL with the
 *    limit named by rks_last_error (split the call).
 *  - The first call on a device does the set-up (the address lookup of the
 *    static array, with that device made current for the call); make it
 *    before any stream capture on that device.
 *  - The scratch is shared by every call in the process on that device:
 *    overlapping calls would race on it, so the library serialises the calls
 *    of one device with a lock (a second thread waits for the first call to
 *    return, also when that call failed part way); calls on different
 *    devices do not wait for each other.
 *  - Nothing needs to start at zero; the call is synchronous (returns with
 *    the outputs in the caller's host arrays). */
#define RKS_XC_NOALLOC_MAX 65536
int rks_eval_xc_noalloc(rks_ctx *ctx, int32_t n, const double *rho, const double *sigma, double *e,
                        double *v_rho, double *v_sigma, int32_t precision);

#ifdef __cplusplus
}
#endif
#endif /* RKS_H */
