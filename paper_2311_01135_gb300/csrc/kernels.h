// Launch wrappers of the device kernels (host side, internal).
#pragma once
#include "common.cuh"

void launch_boys_table(double *t64, float *t32, cudaStream_t s);
void launch_boys_eval(int mmax, int n, const double *dT, double *dout, int fp32, const double *t64,
                      const float *t32, cudaStream_t s);
void launch_quad_tables(double *rad, double *ang, int n_rad, int n_theta, int n_phi, cudaStream_t s);
void launch_onee(const DevBatch &b, int ncand, cudaStream_t s);
void launch_schwarz(const DevBatch &b, int ncand, cudaStream_t s);
void launch_compact_pairs(const DevBatch &b, cudaStream_t s);
void launch_row_count(const DevBatch &b, int ncand, cudaStream_t s);
void launch_row_scan(const DevBatch &b, cudaStream_t s);
void launch_pair_prim(const DevBatch &b, int ncand, int fp32, cudaStream_t s);
void launch_eri_store(const DevBatch &b, int ncand, int fp32, cudaStream_t s);
int launch_grid_build(const DevBatch &b, long long nblk_total, const int *blk_mol, const double *rad,
                      const double *ang, int max_atoms, cudaStream_t s);
// J/K from the packed store.  acc_fp64: accumulate in FP64 (accd) instead of
// FP32 (accf); mode 0: molecules still iterating, 1: every molecule.
// max_pair: largest candidate-pair count of a molecule (sizes the shared pair table).
// Returns -1 when a molecule of max_nbf does not fit the kernel's shared memory.
int launch_jk(const DevBatch &b, int nchunk, int acc_fp64, int mode, int max_nbf, int max_pair, cudaStream_t s);
// Final-step correction of the FP32 store: per-molecule class lists of the
// quartets with Q_pq Q_rs >= fix_theta (built once at setup); in the final
// step one thread per listed quartet recomputes it in FP64 and contracts
// (I64 - I32) with D into the FP64 accumulators.
void launch_fix_list(const DevBatch &b, cudaStream_t s);
// mlist (nlist molecules, nchunk blocks each): only those molecules (the
// precise reruns); null: every molecule (active ones when mode 0), 8 blocks each.
void launch_jk_fix(const DevBatch &b, int mode, cudaStream_t s, const int *mlist = nullptr, int nlist = 0,
                   int nchunk = 8);
// AO + density + B3LYP + V_xc on the grid; acc_fp64 and mode as above.
// skip_tc: leave out the molecules the tensor-core kernel takes (MolDesc::tcq).
void launch_grid_xc(const DevBatch &b, int nchunk, int acc_fp64, int mode, int skip_tc, int max_nbf, int max_nsh,
                    cudaStream_t s);
// Per-block atom significance masks of the tensor-core grid kernel (setup,
// after the grid is built; molecules the kernel does not take are skipped).
void launch_grid_masks(const DevBatch &b, long long nblk_total, const int *blk_mol, cudaStream_t s);
// Tensor-core (tcgen05, 3xTF32) version for the mixed path; takes the
// molecules with a column plan (MolDesc::tcq) and skips the others.
// acc_fp64 = 1 is the final step: density contraction on the CUDA cores
// (round-to-nearest sums).  Molecules the kernel takes, by column class
// (NQ = 4, 8, 12, 16, 20): device list of molecule indices, class offsets and
// counts.
struct TcClasses {
    const int *list;
    int off[5], count[5];
};
void launch_grid_xc_tc(const DevBatch &b, int nchunk, int acc_fp64, int mode, const TcClasses &cl, cudaStream_t s);
// Molecules above RKS_NBF_SMALL (large.cu): J/K with D and the accumulators
// in global memory.  jk_fin: the mixed path's final-step precision; direct:
// every molecule, each quartet recomputed (no store).  Returns -1 when the
// FP64 pair data a direct final step needs is missing.
int launch_jk_large(const DevBatch &b, int nchunk, int jk_fin, int mode, int direct, cudaStream_t s);
// The two-pass grid quadrature of those molecules (b.gcf holds the per-point
// coefficients between the passes); max_nbf / max_nsh over them.  Returns -1
// when their shared memory would not fit.
int launch_grid_xc_large(const DevBatch &b, int nchunk, int acc_fp64, int mode, int max_nbf, int max_nsh,
                         cudaStream_t s);
// Per-molecule FP64 SCF stages.  max_nbf: the largest basis whose matrices
// the kernels keep in shared memory; larger molecules use global scratch.
void launch_scf_init(const DevBatch &b, cudaStream_t s);
// only_rechecked: guess only for the molecules marked by launch_mark_recheck
void launch_scf_guess(const DevBatch &b, int max_nbf, int only_rechecked, cudaStream_t s);
// Fixed protocol, after the iterations: molecules whose DIIS error exceeds
// recheck_fp64_err (or whose status is not OK) are marked for the FP64 redo
// (rechecked = 2, inactive; their indices appended to list); those above
// recheck_err are reset to iterate again from the initial guess (active,
// rechecked = 1); the others become inactive.  counts[0] / counts[1] get the
// number of each; list (FP64 redo) and list1 (precise rerun, any order) have
// room for every molecule.
void launch_mark_recheck(const DevBatch &b, int *counts, int *list, int *list1, cudaStream_t s);
// Results of the FP64 redo: child molecule k replaces parent molecule map[k]
// (state, orbital energies, output density); marks it rechecked = 2.
void launch_adopt(const DevBatch &parent, const DevBatch &child, const int *map, int nchild, cudaStream_t s);
void launch_scf_step(const DevBatch &b, int acc_fp64, int max_nbf, cudaStream_t s);
void launch_scf_final(const DevBatch &b, int acc_fp64, int max_nbf, cudaStream_t s);
void launch_fock_only(const DevBatch &b, int acc_fp64, cudaStream_t s);
void launch_reset_exc(const DevBatch &b, cudaStream_t s);
void launch_count_active(const DevBatch &b, int *out, cudaStream_t s);
void launch_eval_xc(int n, const double *rho, const double *sigma, double *out, int fp32, cudaStream_t s);
// Waits on an mbarrier that is never arrived at, `spins` bounded polls; *gave_up = 1 on expiry.
void launch_wait_selftest(int *gave_up, int spins, cudaStream_t s);
// Peak-rate probe (probe.cu): operations per second of one RKS_PROBE_* kind.
int probe_rate(int kind, cudaStream_t s, double *ops_per_s);
