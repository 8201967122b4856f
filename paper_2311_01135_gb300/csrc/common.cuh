// Internal structures shared by the kernels and the host engine.
//
// One batch = a set of molecules ("slots") resident in HBM.  Every per-molecule
// array lives in a batch-wide buffer; MolDesc holds the offsets.  Kernels take
// a DevBatch by value and index through the descriptors, so one launch covers
// every molecule of the batch (uneven basis sizes included).
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#define RKS_NBF_CAP 224     // largest nbf the kernels are compiled for
#define RKS_NBF_SMALL 96    // largest nbf of the shared-memory J/K, grid and SCF kernels; larger
                            // molecules take the global-memory kernels of large.cu
#define RKS_DIIS_MAX 8
#define RKS_MAXP 3          // primitives per STO-3G shell
#define RKS_PTS_BLOCK 128   // grid points are stored in blocks of this many
#define RKS_NHIST 64        // energies kept per molecule (paper's std(E[-5:]) flag)
#define RKS_FIX_CAP 16384   // FP64-recompute list capacity per molecule and quartet class

// Slot (per-molecule) descriptor.  All offsets are element offsets into the
// batch-wide arrays named in the comments.
struct MolDesc {
    int natom, nbf, nocc, nsh;
    int atom0;          // Z[], axyz[]
    int sh0;            // shell arrays
    int npair_all;      // candidate shell pairs (P >= Q)
    int pair0;          // cand[], cand_q[], kpair[], kq[], row_nq[]; row_off[] uses pair0 + index_in_batch
    int npts;           // real grid points
    int nblk;           // 128-point blocks (padded)
    long long pts0;     // grid arrays (multiple of 128)
    long long eri0;     // packed store (elements)
    long long eri_cap;  // store capacity (unscreened upper bound, elements)
    long long mat0;     // FP64 matrix arena (doubles); see MatSlot
    long long acc0;     // accumulator arena offset (elements), 3 * nbf^2
    int tcq;            // tensor-core grid kernel: columns per quarter NQ (0: CUDA-core kernel)
    int big;            // nbf > RKS_NBF_SMALL: the global-memory kernels of large.cu
};

// FP64 matrices of one molecule, each nbf*nbf, at mat0 + slot * nbf*nbf.
enum MatSlot {
    M_S = 0, M_T, M_V, M_H, M_X, M_D, M_F, M_C, M_J, M_K, M_VXC, M_FX, M_TMP1, M_TMP2, M_TMP3,
    M_DIIS_F, // RKS_DIIS_MAX matrices
    M_DIIS_E = M_DIIS_F + RKS_DIIS_MAX,
    M_COUNT = M_DIIS_E + RKS_DIIS_MAX
};

// Per-molecule FP64 scalars and small state (one struct per slot, device).
struct MolState {
    double E, E_prev, Exc, Enuc, max_err, smin;
    long long exc_fx;       // E_xc accumulator of the current grid pass, fixed point (RKS_FX_EXC)
    double eps_homo, eps_lumo;
    double B[RKS_DIIS_MAX * RKS_DIIS_MAX]; // DIIS Gram matrix of the stored error vectors
    double Ehist[RKS_NHIST];
    int diis_n, diis_head;  // ring buffer: entries, index of the oldest
    int iter;               // SCF iterations done
    int active;             // 1 while iterating
    int converged;
    int status;             // RKS_STATUS_*
    int eigh_fail;
    int c_valid;            // M_C holds the previous step's coefficients (warm-started diagonalisation)
    int err_flag;           // device-side bounds / consistency failures
    int n_quartets;
    int near_ties;
    int rechecked;          // fixed protocol: 1 run again at the final step's precision, 2 redone in FP64
    long long n_elem;       // store elements written
    double grid_pairs[2];   // sum over grid blocks of 128 n_sig^2 (n_sig: AOs significant in the
                            // block), iterations / final step: the screened work of one grid pass
    double eps[RKS_NBF_CAP];
};

// Fixed-point accumulator: the value times 2^40 in a 64-bit integer.  Integer
// atomic adds are associative, so a sum does not depend on the order in which
// threads, warps or blocks arrive: the mixed-precision iterations of a
// molecule give the same bits alone or in any batch.  Range +-8.4e6, step
// 9.1e-13; each FP32 contribution is rounded once to the step.
struct Fx {
    long long v;
};
#define RKS_FX_SCALE 1099511627776.0         // 2^40
#define RKS_FX_EXC 17592186044416.0          // 2^44: E_xc partial sums (|E_xc| < 5e5 Ha)
__device__ __forceinline__ void acc_add(float *p, float x) { atomicAdd(p, x); }
__device__ __forceinline__ void acc_add(double *p, double x) { atomicAdd(p, x); }
__device__ __forceinline__ void acc_add(Fx *p, float x) {
    atomicAdd((unsigned long long *)&p->v, (unsigned long long)__float2ll_rn(x * (float)RKS_FX_SCALE));
}
__device__ __forceinline__ void acc_add(Fx *p, double x) {
    atomicAdd((unsigned long long *)&p->v, (unsigned long long)__double2ll_rn(x * RKS_FX_SCALE));
}
__host__ __device__ __forceinline__ double acc_value(float x) { return (double)x; }
__host__ __device__ __forceinline__ double acc_value(double x) { return x; }
__host__ __device__ __forceinline__ double acc_value(Fx x) { return (double)x.v * (1.0 / RKS_FX_SCALE); }
// merging a block's shared-memory partial sums into the global accumulators
__device__ __forceinline__ bool acc_nonzero(double x) { return x != 0.0; }
__device__ __forceinline__ bool acc_nonzero(Fx x) { return x.v != 0; }
__device__ __forceinline__ void acc_merge(double *p, double x) { atomicAdd(p, x); }
__device__ __forceinline__ void acc_merge(Fx *p, Fx x) {
    atomicAdd((unsigned long long *)&p->v, (unsigned long long)x.v);
}
// E_xc partials (one per warp) into the molecule's fixed-point E_xc
__device__ __forceinline__ void exc_add(long long *p, double x) {
    atomicAdd((unsigned long long *)p, (unsigned long long)__double2ll_rn(x * RKS_FX_EXC));
}

// The tensor-core grid kernel's column plan (one per molecule it takes; the
// choice is made per molecule, so a molecule runs the same arithmetic
// whatever else is in its batch).  Its threads own AO columns in four
// quarters of NQ = 4, 8, 12, 16 or 20 (padded basis 4 NQ <= 80); a quarter is
// NQ / 5 units of five columns and NQ % 5 single columns.  A unit holds one
// heavy atom (1s, 2s, 2px, 2py, 2pz: STO-3G for C, N, O, F, with the 2s and
// 2p shells sharing exponents) or up to five hydrogens; a single column holds
// one hydrogen.  Per molecule, RKS_TC_PLAN ints:
//   [q * 5 + k], k < NQ / 5: unit word of quarter q: bit 31 heavy; atom ids
//                             in 6-bit fields (field r = slot r; 63 = empty)
//   [q * 5 + 4]:             the single columns' atom ids, same fields
//   [20 + c], c < 80:        AO index of the kernel's column c (-1: padding)
#define RKS_TC_NPMAX 80
#define RKS_TC_NATMAX 63
#define RKS_TC_PLAN 100
#define RKS_TC_EMPTY 63

// Device view of a batch (passed by value to kernels).
struct DevBatch {
    int nmol;
    int precision;          // 0 FP64, 1 mixed
    int xc;                 // 1 B3LYP, 0 Hartree-Fock
    double a0;              // exact-exchange fraction in the Fock matrix
    const MolDesc *mol;
    MolState *st;
    // atoms
    const int *Z;
    const double *axyz;     // [natom][3]
    // shells in packing order (s shells, then p shells; atom order inside)
    const int *sh_atom, *sh_l, *sh_ao0;
    const double *sh_xyz;   // [nsh][3]
    const double *sh_ex;    // [nsh][3]
    const double *sh_co;    // [nsh][3] normalised contraction coefficients
    // candidate shell pairs (all P >= Q, ordered by (l_P + l_Q, P, Q))
    const int2 *cand;
    const int *cand_mol;    // owning molecule of each candidate
    double *cand_q;         // Schwarz Q per candidate
    int2 *kpair;            // kept pairs (compacted, same order)
    double *kq;             // their Q
    int *npair;             // kept pairs per molecule
    int *row_nq;            // kept quartets per kept row
    long long *row_off;     // exclusive prefix of row element counts; [pair0 + m + r], r <= npair
    void *store;            // packed ERIs (float or double)
    void *pairprim;         // per kept pair: 9 primitive-pair records (K, zeta, P - A), float or double
    void *pairprim64;       // FP64 copy for the final-step FP64 recompute of the mixed path (or null)
    int4 *fixlist;          // per molecule, per quartet class: (row, col, store offset lo, hi) of quartets
                            // with Q_pq Q_rs >= fix_theta; RKS_FIX_CAP entries per class
    int *fixcount;          // [nmol][6] entries written (may exceed the capacity: then capped)
    double fix_theta;
    // grid (SoA, padded blocks; padding points have w = 0)
    void *gx, *gy, *gz, *gw;
    // per 128-point block: atoms with a shell significant in it, bit per
    // atom, [2 * block] iterations, [2 * block + 1] final step; filled for the
    // molecules the tensor-core grid kernel takes (mixed path), else null
    unsigned long long *blk_mask;
    const int *tc_plan;     // [nmol][RKS_TC_PLAN] column plans (mixed path), else null
    // FP64 matrices
    double *mat;
    // accumulators J', K', V' (3 * nbf^2 per molecule at acc0): 64-bit fixed
    // point in every pass of the mixed path (accx), FP64 for the FP64 path
    // (accd); both views share one buffer, zeroed before each pass
    struct Fx *accx;
    double *accd;
    int *jk_next;           // [nmol] J/K row queue heads (zeroed before each J/K launch)
    void *gcf;              // molecules above RKS_NBF_SMALL: per grid point the four coefficients of
                            // X (w v_rho / 2, 2 w v_sigma grad rho), [pts0 + p][4] (T), else null
    int direct;             // 1: no packed store; J/K recompute the quartets every pass (direct SCF)
    void *gdt;              // mixed path, molecules above RKS_NBF_SMALL: D in FP32 for the grid
                            // pass, n^2 floats at acc0 (converted once per pass), else null
    // Boys tables
    const double *boys64;
    const float *boys32;
    // grid options
    int n_rad, n_theta, n_phi, becke_iters;
    int diis_space;
    int fixed_iters, max_iters;
    int guess;              // 0 superposed atoms, 1 core Hamiltonian
    double e_tol, err_tol;
    double recheck_err;     // fixed protocol: DIIS error above which a molecule is run again
    double recheck_fp64_err; // and above which it is redone on the FP64 path
};

__host__ __device__ inline long long nbf2(int n) { return (long long)n * n; }

__device__ inline double *matp(const DevBatch &b, const MolDesc &m, int slot) {
    return b.mat + m.mat0 + (long long)slot * nbf2(m.nbf);
}

// Boys table layout: rows T_i = i * h for i = 0..n-1, columns F_0..F_(ncol-1).
#define BOYS_H 0.05
#define BOYS_N64 801   // T < 40 in FP64 (Taylor, 7 terms)
#define BOYS_COL64 11
#define BOYS_TMAX64 40.0
#define BOYS_N32 601   // T < 30 in FP32 (Taylor, 4 terms)
#define BOYS_COL32 8
#define BOYS_TMAX32 30.0

#define CUDA_OK(x)                                                                              \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess) return rks_cuda_fail(e_, #x, __FILE__, __LINE__);                \
    } while (0)

int rks_cuda_fail(cudaError_t e, const char *what, const char *file, int line);
