// Per-molecule FP64 SCF stages, one thread block per molecule.
//
// Paper Section 3.1 (Eq. 1): at iteration i, build rho_i, V_xc, J, K, then
// solve [V + T + J + K + V_xc] C = S C eps for the next C.  Readings (the paper
// is silent on them):
//  * F = H + J - (a0/2) K_std + V_xc, a0 = 0.2 for B3LYP (1 in Hartree-Fock mode);
//  * E = tr D (H + J/2 - a0 K_std/4) + E_xc + E_nuc;
//  * X = S^-1/2 (Loewdin), X^T F X diagonalised by Jacobi, C = X C' (after the
//    first step in the previous step's MO basis: C_prev^T F C_prev, C = C_prev V);
//  * initial density from superposed neutral atoms (default) or the core Hamiltonian;
//  * Pulay DIIS on e = X^T (F D S - S D F) X with the last diis_space pairs,
//    used once two pairs exist; a singular bordered system drops the oldest pair;
//  * convergence: |E - E_prev| < e_tol and max|e| < err_tol (converge protocol),
//    or exactly fixed_iters iterations; then one plain final Fock build.
#include <cfloat>

#include "common.cuh"
#include "kernels.h"
#include "la.cuh"

#define RKS_STATUS_OK_ 0
#define RKS_STATUS_NOT_CONVERGED_ 1
#define RKS_STATUS_NONFINITE_ 2
#define RKS_STATUS_S_ILL_ 3
#define RKS_STATUS_EIGH_ 4

struct ScfSmem {
    double *A, *V, *w, *red, *cs;
    int *perm;
};

// A and V are sized for the batch's largest basis nmax (not the compiled
// cap), so that two or three molecules' blocks share an SM: the step is
// latency-bound FP64 work and gains from the extra resident warps.  A
// molecule above nmax (a basis above RKS_NBF_SMALL: 2 n^2 doubles exceed
// shared memory) keeps A and V in its global scratch matrices M_TMP2 and
// M_TMP3 instead (scf_big_scratch); every caller leaves those two free while
// it diagonalises.
__device__ inline ScfSmem scf_smem(unsigned char *raw, int nmax) {
    ScfSmem s;
    double *d = (double *)raw;
    s.A = d;
    s.V = d + nmax * nmax;
    s.w = s.V + nmax * nmax;
    s.red = s.w + RKS_NBF_CAP;
    s.cs = s.red + 64;
    s.perm = (int *)(s.cs + 2 * RKS_NBF_CAP + 8);
    return s;
}
__device__ inline void scf_big_scratch(ScfSmem &sm, const DevBatch &b, const MolDesc &md, int nmax) {
    if (md.nbf > nmax) {
        const long long nn = nbf2(md.nbf);
        sm.A = b.mat + md.mat0 + (long long)M_TMP2 * nn;
        sm.V = b.mat + md.mat0 + (long long)M_TMP3 * nn;
    }
}
static size_t scf_smem_bytes(int nmax) {
    return sizeof(double) * (2 * (size_t)nmax * nmax + RKS_NBF_CAP + 64 + 2 * RKS_NBF_CAP + 8) +
           sizeof(int) * (3 * RKS_NBF_CAP + 8);
}

// Diagonalise F in the Loewdin basis: eigenvalues -> w (shared), C = X C'
// (global, in/out).
// Cold start: Jacobi on X^T F X, then C = X V.
// Warm start (C holds the previous step's coefficients, so C^T S C = I):
// Jacobi on C^T F C, which is X^T F X in the previous eigenvector basis and
// nearly diagonal after the first SCF iterations, then C <- C V.  This is
// the cold form with C' = C'_prev V, for half the FP64 products.
__device__ int diag_fock(const double *F, const double *X, double *tmp, double *C, ScfSmem &sm, int n, bool warm) {
    const double *B = warm ? C : X;
    la::gemm(tmp, F, B, n, false, false);
    __syncthreads();
    la::gemm(sm.A, B, tmp, n, true, false);
    __syncthreads();
    int sw = la::jacobi(sm.A, sm.V, sm.w, n, sm.red, sm.perm, sm.cs);
    la::gemm(tmp, B, sm.V, n, false, false);
    __syncthreads();
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) C[i] = tmp[i];
    __syncthreads();
    return sw;
}

__device__ void density_from_C(const double *C, double *D, int n, int nocc) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        int i = idx / n, j = idx % n;
        double s = 0.0;
        for (int k = 0; k < nocc; k++) s += C[i * n + k] * C[j * n + k];
        D[idx] = 2.0 * s;
    }
    __syncthreads();
}

// ------------------------------------------------------------------ init
__global__ void scf_init_kernel(DevBatch b) {
    const int m = blockIdx.x;
    const MolDesc md = b.mol[m];
    const int n = md.nbf, nn = n * n;
    double *Tm = b.mat + md.mat0 + (long long)M_T * nn, *Vm = b.mat + md.mat0 + (long long)M_V * nn;
    double *H = b.mat + md.mat0 + (long long)M_H * nn;
    for (int i = threadIdx.x; i < nn; i += blockDim.x) H[i] = Tm[i] + Vm[i];
    __shared__ double red[32];
    double e = 0.0;
    for (int idx = threadIdx.x; idx < md.natom * md.natom; idx += blockDim.x) {
        int a = idx / md.natom, c = idx % md.natom;
        if (c < a) {
            const double *xa = b.axyz + (md.atom0 + a) * 3, *xc = b.axyz + (md.atom0 + c) * 3;
            double dx = xa[0] - xc[0], dy = xa[1] - xc[1], dz = xa[2] - xc[2];
            e += (double)b.Z[md.atom0 + a] * b.Z[md.atom0 + c] / sqrt(dx * dx + dy * dy + dz * dz);
        }
    }
    e = la::block_sum(e, red);
    if (threadIdx.x == 0) {
        MolState &st = b.st[m];
        st.Enuc = e;
        st.E = 0.0; st.E_prev = 0.0; st.Exc = 0.0; st.max_err = 0.0;
        st.diis_n = 0; st.diis_head = 0; st.iter = 0; st.active = 1; st.converged = 0;
        st.status = RKS_STATUS_OK_; st.eigh_fail = 0; st.c_valid = 0; st.rechecked = 0;
    }
}

void launch_scf_init(const DevBatch &b, cudaStream_t s) { scf_init_kernel<<<b.nmol, 256, 0, s>>>(b); }

// ------------------------------------------- orthogonaliser + core guess
__global__ void scf_guess_kernel(DevBatch b, int nmax, int only_rechecked) {
    extern __shared__ unsigned char raw[];
    ScfSmem sm = scf_smem(raw, nmax);
    const int m = blockIdx.x;
    if (only_rechecked && !b.st[m].rechecked) return;
    const MolDesc md = b.mol[m];
    scf_big_scratch(sm, b, md, nmax);
    const int n = md.nbf, nn = n * n;
    double *S = b.mat + md.mat0 + (long long)M_S * nn;
    double *X = b.mat + md.mat0 + (long long)M_X * nn;
    double *H = b.mat + md.mat0 + (long long)M_H * nn;
    double *C = b.mat + md.mat0 + (long long)M_C * nn;
    double *D = b.mat + md.mat0 + (long long)M_D * nn;
    double *tmp = b.mat + md.mat0 + (long long)M_TMP1 * nn;
    for (int i = threadIdx.x; i < nn; i += blockDim.x) sm.A[i] = S[i];
    __syncthreads();
    int sw = la::jacobi(sm.A, sm.V, sm.w, n, sm.red, sm.perm, sm.cs);
    // X = U diag(s^-1/2) U^T
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
        int i = idx / n, j = idx % n;
        double v = 0.0;
        for (int k = 0; k < n; k++) v += sm.V[i * n + k] * sm.V[j * n + k] / sqrt(sm.w[k]);
        X[idx] = v;
    }
    __syncthreads();
    double smin = sm.w[0];
    int sw2 = 0;
    if (b.guess == 1) {
        // core Hamiltonian: diagonalise X^T H X, occupy the lowest n_occ
        sw2 = diag_fock(H, X, tmp, C, sm, n, false);
        density_from_C(C, D, n, md.nocc);
    } else {
        // superposed neutral atoms: per heavy atom D_ss = 2 S_ss^-1 over (1s, 2s)
        // and (Z - 4)/3 on each 2p; per H 1/S_11; zero between atoms
        for (int i = threadIdx.x; i < nn; i += blockDim.x) D[i] = 0.0;
        __syncthreads();
        if (threadIdx.x == 0) {
            int i = 0;
            for (int a = 0; a < md.natom; a++) {
                const int z = b.Z[md.atom0 + a];
                if (z == 1) {
                    D[i * n + i] = 1.0 / S[i * n + i];
                    i += 1;
                    continue;
                }
                const double s00 = S[i * n + i], s01 = S[i * n + i + 1], s11 = S[(i + 1) * n + i + 1];
                const double det = s00 * s11 - s01 * s01;
                D[i * n + i] = 2.0 * s11 / det;
                D[i * n + i + 1] = D[(i + 1) * n + i] = -2.0 * s01 / det;
                D[(i + 1) * n + i + 1] = 2.0 * s00 / det;
                for (int k = 2; k < 5; k++) D[(i + k) * n + i + k] = (z - 4) / 3.0;
                i += 5;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        MolState &st = b.st[m];
        st.smin = smin;
        if (smin < 1e-8) st.status = RKS_STATUS_S_ILL_;
        if (sw < 0 || sw2 < 0) st.eigh_fail++;
        for (int i = 0; i < n; i++) st.eps[i] = sm.w[i];
        st.c_valid = (b.guess == 1);
    }
}

void launch_scf_guess(const DevBatch &b, int max_nbf, int only_rechecked, cudaStream_t s) {
    const size_t sm = scf_smem_bytes(max_nbf);
    cudaFuncSetAttribute(scf_guess_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    scf_guess_kernel<<<b.nmol, 256, sm, s>>>(b, max_nbf, only_rechecked);
}

// Fixed protocol: after the iterations, a molecule still far from its fixed
// point (DIIS error above recheck_err) has an energy E[D_n] that is not
// stationary, so it depends on the path of the iterations and the FP32
// rounding of the mixed Fock builds steers it.  Such molecules start again
// from the initial guess (fresh DIIS history, same iteration count) with
// every Fock build at the final step's precision.  Molecules that have not
// converged at all (DIIS error above recheck_fp64_err, or a bad status) are
// redone on the FP64 path: there the path is sensitive to rounding far below
// FP32 (paper Section 3.2, "Numerical Error": the float32 results are taken
// for the converged ~99%, the rest recomputed in float64).  The rest wait for
// the final step.  The decision reads only the molecule's own state.
__global__ void mark_recheck_kernel(DevBatch b, int *counts, int *list, int *list1) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < b.nmol; m += gridDim.x * blockDim.x) {
        MolState &st = b.st[m];
        const bool bad = st.status != RKS_STATUS_OK_ || !(st.max_err <= b.recheck_fp64_err);
        const bool fp64 = !st.rechecked && st.status != RKS_STATUS_S_ILL_ && b.recheck_fp64_err > 0.0 && bad;
        const bool again = !st.rechecked && !fp64 && st.status != RKS_STATUS_S_ILL_ &&
                           (st.status != RKS_STATUS_OK_ || !(st.max_err <= b.recheck_err));
        if (fp64) {
            st.rechecked = 2;
            st.active = 0;
            list[atomicAdd(&counts[1], 1)] = m;
        } else if (again) {
            list1[atomicAdd(&counts[0], 1)] = m;
            st.rechecked = 1;
            st.active = 1;
            st.iter = 0;
            st.diis_n = 0;
            st.diis_head = 0;
            st.E = 0.0;
            st.E_prev = 0.0;
            st.max_err = 0.0;
            st.status = RKS_STATUS_OK_;
            st.eigh_fail = 0;
            st.c_valid = 0;
        } else {
            st.active = 0;
        }
    }
}

void launch_mark_recheck(const DevBatch &b, int *counts, int *list, int *list1, cudaStream_t s) {
    cudaMemsetAsync(counts, 0, 2 * sizeof(int), s);
    mark_recheck_kernel<<<(b.nmol + 255) / 256, 256, 0, s>>>(b, counts, list, list1);
}

// One block per redone molecule: its FP64 state and output density replace
// the parent's (the parent's own final step for it is discarded).
__global__ void adopt_kernel(DevBatch parent, DevBatch child, const int *map) {
    const int k = blockIdx.x, m = map[k];
    const MolDesc mp = parent.mol[m], mc = child.mol[k];
    const long long nn = nbf2(mp.nbf);
    const double *src = child.mat + mc.mat0 + (long long)M_D * nn;
    double *dst = parent.mat + mp.mat0 + (long long)M_D * nn;
    for (long long i = threadIdx.x; i < nn; i += blockDim.x) dst[i] = src[i];
    const int words = (int)(sizeof(MolState) / sizeof(int));
    const int *s = (const int *)(child.st + k);
    int *d = (int *)(parent.st + m);
    for (int i = threadIdx.x; i < words; i += blockDim.x) d[i] = s[i];
    __syncthreads();
    if (threadIdx.x == 0) parent.st[m].rechecked = 2;
}

void launch_adopt(const DevBatch &parent, const DevBatch &child, const int *map, int nchild, cudaStream_t s) {
    if (nchild > 0) adopt_kernel<<<nchild, 256, 0, s>>>(parent, child, map);
}

// ----------------------------------------------------- Fock assembly
// J = J' + J'^T etc. from the accumulators; F = H + J - a0/2 K + V_xc;
// returns E (valid in every thread).
template <typename TA>
__device__ double assemble_fock(const DevBatch &b, int m, const MolDesc &md, const TA *acc, double *red) {
    const int n = md.nbf, nn = n * n;
    double *H = b.mat + md.mat0 + (long long)M_H * nn;
    double *D = b.mat + md.mat0 + (long long)M_D * nn;
    double *F = b.mat + md.mat0 + (long long)M_F * nn;
    double *J = b.mat + md.mat0 + (long long)M_J * nn;
    double *K = b.mat + md.mat0 + (long long)M_K * nn;
    double *Vx = b.mat + md.mat0 + (long long)M_VXC * nn;
    const TA *aJ = acc, *aK = acc + nn, *aV = acc + 2 * nn;
    double e = 0.0;
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
        int i = idx / n, j = idx % n, tr = j * n + i;
        double jj = acc_value(aJ[idx]) + acc_value(aJ[tr]);
        double kk = acc_value(aK[idx]) + acc_value(aK[tr]);
        double vv = b.xc ? acc_value(aV[idx]) + acc_value(aV[tr]) : 0.0;
        J[idx] = jj;
        K[idx] = kk;
        Vx[idx] = vv;
        F[idx] = H[idx] + jj - 0.5 * b.a0 * kk + vv;
        e += D[idx] * (H[idx] + 0.5 * jj - 0.25 * b.a0 * kk);
    }
    e = la::block_sum(e, red);
    const double exc = (double)b.st[m].exc_fx * (1.0 / RKS_FX_EXC);
    __syncthreads();
    if (threadIdx.x == 0) b.st[m].Exc = exc;
    return e + exc + b.st[m].Enuc;
}

// ------------------------------------------------------------ one step
template <typename TA>
__global__ void scf_step_kernel(DevBatch b, const TA *accbase, int nmax) {
    extern __shared__ unsigned char raw[];
    ScfSmem sm = scf_smem(raw, nmax);
    const int m = blockIdx.x;
    const MolDesc &md = b.mol[m];
    MolState &st = b.st[m];
    if (!st.active) return;
    scf_big_scratch(sm, b, md, nmax);
    const int n = md.nbf, nn = n * n;
    double *S = b.mat + md.mat0 + (long long)M_S * nn;
    double *X = b.mat + md.mat0 + (long long)M_X * nn;
    double *D = b.mat + md.mat0 + (long long)M_D * nn;
    double *F = b.mat + md.mat0 + (long long)M_F * nn;
    double *C = b.mat + md.mat0 + (long long)M_C * nn;
    double *FX = b.mat + md.mat0 + (long long)M_FX * nn;
    double *t1 = b.mat + md.mat0 + (long long)M_TMP1 * nn;
    double *t2 = b.mat + md.mat0 + (long long)M_TMP2 * nn;
    double *t3 = b.mat + md.mat0 + (long long)M_TMP3 * nn;
    const double E = assemble_fock<TA>(b, m, md, accbase + md.acc0, sm.red);
    __syncthreads();
    // e = X^T (F D S - S D F) X ;  S D F = (F D S)^T for symmetric F, D, S
    la::gemm(t1, F, D, n, false, false);
    __syncthreads();
    la::gemm(t2, t1, S, n, false, false);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
        int i = idx / n, j = idx % n;
        t3[idx] = t2[idx] - t2[j * n + i];
    }
    __syncthreads();
    la::gemm(t1, X, t3, n, true, false);
    __syncthreads();
    la::gemm(t2, t1, X, n, false, false);  // t2 = error matrix
    __syncthreads();
    double mx = 0.0;
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) mx = fmax(mx, fabs(t2[idx]));
    mx = la::block_max(mx, sm.red);
    const int diis_space = b.diis_space;
    __shared__ int s_conv, s_nd, s_ok;
    __shared__ double s_c[RKS_DIIS_MAX + 1];
    __shared__ int s_slot[RKS_DIIS_MAX];
    if (threadIdx.x == 0) {
        s_conv = 0;
        if (!isfinite(E) || !isfinite(mx)) {
            st.status = RKS_STATUS_NONFINITE_;
            st.active = 0;
            s_conv = 2;
        } else if (b.fixed_iters == 0 && st.iter >= 1 && fabs(E - st.E_prev) < b.e_tol && mx < b.err_tol) {
            st.converged = 1;
            st.active = 0;
            s_conv = 1;
        }
        st.E = E;
        st.max_err = mx;
        st.Ehist[st.iter % RKS_NHIST] = E;
    }
    __syncthreads();
    if (s_conv) {
        if (threadIdx.x == 0) st.iter += 1;
        return;
    }
    // ---- DIIS push
    __shared__ int s_new;
    if (threadIdx.x == 0) {
        int slot;
        if (st.diis_n < diis_space) {
            slot = (st.diis_head + st.diis_n) % diis_space;
            st.diis_n++;
        } else {
            slot = st.diis_head;
            st.diis_head = (st.diis_head + 1) % diis_space;
        }
        s_new = slot;
    }
    __syncthreads();
    double *Fh = b.mat + md.mat0 + (long long)(M_DIIS_F + s_new) * nn;
    double *Eh = b.mat + md.mat0 + (long long)(M_DIIS_E + s_new) * nn;
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
        Fh[idx] = F[idx];
        Eh[idx] = t2[idx];
    }
    __syncthreads();
    for (int k = 0; k < st.diis_n; k++) {
        int slot = (st.diis_head + k) % diis_space;
        const double *Ek = b.mat + md.mat0 + (long long)(M_DIIS_E + slot) * nn;
        double d = 0.0;
        for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) d += Eh[idx] * Ek[idx];
        d = la::block_sum(d, sm.red);
        if (threadIdx.x == 0) {
            st.B[s_new * RKS_DIIS_MAX + slot] = d;
            st.B[slot * RKS_DIIS_MAX + s_new] = d;
        }
    }
    __syncthreads();
    // ---- DIIS solve (thread 0): bordered system, oldest -> newest
    if (threadIdx.x == 0) {
        s_ok = 0;
        while (st.diis_n >= 2) {
            int mm = st.diis_n;
            double Mtx[(RKS_DIIS_MAX + 1) * (RKS_DIIS_MAX + 2)];
            const int W = mm + 2;
            for (int i = 0; i < mm; i++) {
                int si = (st.diis_head + i) % diis_space;
                s_slot[i] = si;
                for (int j = 0; j < mm; j++) {
                    int sj = (st.diis_head + j) % diis_space;
                    Mtx[i * W + j] = st.B[si * RKS_DIIS_MAX + sj];
                }
                Mtx[i * W + mm] = -1.0;
                Mtx[i * W + mm + 1] = 0.0;
            }
            for (int j = 0; j < mm; j++) Mtx[mm * W + j] = -1.0;
            Mtx[mm * W + mm] = 0.0;
            Mtx[mm * W + mm + 1] = -1.0;
            bool sing = false;
            const int N = mm + 1;
            for (int c = 0; c < N && !sing; c++) {
                int piv = c;
                for (int r = c + 1; r < N; r++)
                    if (fabs(Mtx[r * W + c]) > fabs(Mtx[piv * W + c])) piv = r;
                if (Mtx[piv * W + c] == 0.0) { sing = true; break; }
                if (piv != c)
                    for (int k = 0; k < W; k++) { double t = Mtx[c * W + k]; Mtx[c * W + k] = Mtx[piv * W + k]; Mtx[piv * W + k] = t; }
                for (int r = c + 1; r < N; r++) {
                    double f = Mtx[r * W + c] / Mtx[c * W + c];
                    for (int k = c; k < W; k++) Mtx[r * W + k] -= f * Mtx[c * W + k];
                }
            }
            if (!sing) {
                for (int r = N - 1; r >= 0; r--) {
                    double v = Mtx[r * W + N];
                    for (int k = r + 1; k < N; k++) v -= Mtx[r * W + k] * s_c[k];
                    s_c[r] = v / Mtx[r * W + r];
                }
                bool fin = true;
                for (int i = 0; i < N; i++) fin = fin && isfinite(s_c[i]);
                if (fin) { s_ok = 1; s_nd = mm; break; }
            }
            // drop the oldest pair
            st.diis_head = (st.diis_head + 1) % diis_space;
            st.diis_n--;
        }
    }
    __syncthreads();
    const double *Fuse = F;
    if (s_ok) {
        for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
            double v = 0.0;
            for (int k = 0; k < s_nd; k++) v += s_c[k] * b.mat[md.mat0 + (long long)(M_DIIS_F + s_slot[k]) * nn + idx];
            FX[idx] = v;
        }
        __syncthreads();
        Fuse = FX;
    }
    // ---- diagonalise, new density
    int sw = diag_fock(Fuse, X, t1, C, sm, n, st.c_valid != 0);
    density_from_C(C, D, n, md.nocc);
    if (threadIdx.x == 0) {
        if (sw < 0) st.eigh_fail++;
        st.c_valid = 1;
        st.E_prev = E;
        st.iter += 1;
        for (int i = 0; i < n; i++) st.eps[i] = sm.w[i];
        if (b.fixed_iters > 0 && st.iter >= b.fixed_iters) st.active = 0;
        if (b.fixed_iters == 0 && st.iter >= b.max_iters) {
            st.active = 0;
            st.status = RKS_STATUS_NOT_CONVERGED_;
        }
    }
}

void launch_scf_step(const DevBatch &b, int acc_fp64, int max_nbf, cudaStream_t s) {
    (void)acc_fp64;
    const size_t sm = scf_smem_bytes(max_nbf);
    if (b.precision == 0) {
        cudaFuncSetAttribute(scf_step_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        scf_step_kernel<double><<<b.nmol, 256, sm, s>>>(b, b.accd, max_nbf);
    } else {
        cudaFuncSetAttribute(scf_step_kernel<Fx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        scf_step_kernel<Fx><<<b.nmol, 256, sm, s>>>(b, b.accx, max_nbf);
    }
}

// ------------------------------------------------------------ final
// F[D] at the last density (final precision), E[D], plain diagonalisation:
// eps, HOMO/LUMO, and the output density (written over M_D; the input
// density is kept in M_TMP3).
template <typename TA>
__global__ void scf_final_kernel(DevBatch b, const TA *accbase, int nmax) {
    extern __shared__ unsigned char raw[];
    ScfSmem sm = scf_smem(raw, nmax);
    const int m = blockIdx.x;
    const MolDesc &md = b.mol[m];
    MolState &st = b.st[m];
    scf_big_scratch(sm, b, md, nmax);
    const int n = md.nbf, nn = n * n;
    double *X = b.mat + md.mat0 + (long long)M_X * nn;
    double *D = b.mat + md.mat0 + (long long)M_D * nn;
    double *F = b.mat + md.mat0 + (long long)M_F * nn;
    double *C = b.mat + md.mat0 + (long long)M_C * nn;
    double *t1 = b.mat + md.mat0 + (long long)M_TMP1 * nn;
    double *t3 = b.mat + md.mat0 + (long long)M_TMP3 * nn;
    const double E = assemble_fock<TA>(b, m, md, accbase + md.acc0, sm.red);
    __syncthreads();
    int sw = diag_fock(F, X, t1, C, sm, n, st.c_valid != 0);
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) t3[idx] = D[idx];
    __syncthreads();
    density_from_C(C, D, n, md.nocc);
    if (threadIdx.x == 0) {
        if (sw < 0) st.eigh_fail++;
        st.E = E;
        for (int i = 0; i < n; i++) st.eps[i] = sm.w[i];
        st.eps_homo = sm.w[md.nocc - 1];
        st.eps_lumo = md.nocc < n ? sm.w[md.nocc] : 0.0;
        bool fin = isfinite(E);
        for (int i = 0; i < n; i++) fin = fin && isfinite(sm.w[i]);
        if (!fin) st.status = RKS_STATUS_NONFINITE_;
        else if (st.eigh_fail && st.status == RKS_STATUS_OK_) st.status = RKS_STATUS_EIGH_;
        st.active = 0;
    }
}

void launch_scf_final(const DevBatch &b, int acc_fp64, int max_nbf, cudaStream_t s) {
    (void)acc_fp64;  // the accumulator type follows the precision: FP64 path double, mixed fixed point
    const size_t sm = scf_smem_bytes(max_nbf);
    if (b.precision == 0) {
        cudaFuncSetAttribute(scf_final_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        scf_final_kernel<double><<<b.nmol, 256, sm, s>>>(b, b.accd, max_nbf);
    } else {
        cudaFuncSetAttribute(scf_final_kernel<Fx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        scf_final_kernel<Fx><<<b.nmol, 256, sm, s>>>(b, b.accx, max_nbf);
    }
}

// ---------------------------------------------- Fock build at a given D
template <typename TA>
__global__ void fock_only_kernel(DevBatch b, const TA *accbase) {
    __shared__ double red[32];
    const int m = blockIdx.x;
    const MolDesc &md = b.mol[m];
    const double E = assemble_fock<TA>(b, m, md, accbase + md.acc0, red);
    if (threadIdx.x == 0) b.st[m].E = E;
}

void launch_fock_only(const DevBatch &b, int acc_fp64, cudaStream_t s) {
    (void)acc_fp64;
    if (b.precision == 0) fock_only_kernel<double><<<b.nmol, 256, 0, s>>>(b, b.accd);
    else fock_only_kernel<Fx><<<b.nmol, 256, 0, s>>>(b, b.accx);
}

// Exc accumulators to zero before a grid pass.
__global__ void reset_exc_kernel(DevBatch b) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < b.nmol) {
        b.st[m].Exc = 0.0;
        b.st[m].exc_fx = 0;
    }
}
void launch_reset_exc(const DevBatch &b, cudaStream_t s) {
    reset_exc_kernel<<<(b.nmol + 127) / 128, 128, 0, s>>>(b);
}

// Number of molecules still iterating, for the host's convergence polling
// (one int instead of the whole state array).
__global__ void count_active_kernel(DevBatch b, int *out) {
    __shared__ int tot;
    if (threadIdx.x == 0) tot = 0;
    __syncthreads();
    int n = 0;
    for (int m = threadIdx.x; m < b.nmol; m += blockDim.x) n += b.st[m].active != 0;
    if (n) atomicAdd(&tot, n);
    __syncthreads();
    if (threadIdx.x == 0) *out = tot;
}
void launch_count_active(const DevBatch &b, int *out, cudaStream_t s) {
    count_active_kernel<<<1, 256, 0, s>>>(b, out);
}
