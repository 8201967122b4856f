// FP64 dense linear algebra for one molecule inside one thread block:
// small GEMMs and a parallel-ordering (round-robin) cyclic Jacobi eigensolver.
//
// The paper's iteration solves the generalised eigenproblem F C = S C eps each
// step (Section 3.1, Eq. 1).  Here it becomes a symmetric eigenproblem through
// the Loewdin orthogonaliser X = S^-1/2:  (X^T F X) C' = C' eps, C = X C'.
// Matrices are n x n row-major with leading dimension n (n <= RKS_NBF_CAP).
#pragma once
#include "common.cuh"

namespace la {

// C = alpha * op(A) op(B) + beta * C;  ta/tb: use the transpose.
// Any of the pointers may be shared or global memory.  Caller syncs after.
__device__ inline void gemm(double *C, const double *A, const double *B, int n, bool ta, bool tb,
                            double alpha = 1.0, double beta = 0.0) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        int i = idx / n, j = idx % n;
        double s = 0.0;
        if (!ta && !tb) {
            for (int k = 0; k < n; k++) s += A[i * n + k] * B[k * n + j];
        } else if (ta && !tb) {
            for (int k = 0; k < n; k++) s += A[k * n + i] * B[k * n + j];
        } else if (!ta && tb) {
            for (int k = 0; k < n; k++) s += A[i * n + k] * B[j * n + k];
        } else {
            for (int k = 0; k < n; k++) s += A[k * n + i] * B[j * n + k];
        }
        C[idx] = alpha * s + (beta == 0.0 ? 0.0 : beta * C[idx]);
    }
}

// Block-wide sum of one double per thread (result valid in every thread).
__device__ inline double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; i++) t += red[i];
    __syncthreads();
    return t;
}

__device__ inline double block_max(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = red[0];
    int nw = (blockDim.x + 31) >> 5;
    for (int i = 1; i < nw; i++) t = fmax(t, red[i]);
    __syncthreads();
    return t;
}

// Symmetric eigendecomposition A = V diag(w) V^T by cyclic Jacobi with the
// round-robin ("tournament") ordering: each step applies n/2 disjoint plane
// rotations at once, a sweep has n-1 steps.  Position 0 stays, positions
// 1..ne-1 rotate by one per step; pair k of a step joins positions k and
// ne-1-k.
// Rotation per pair (p, q) (Rutishauser's form): theta = (a_qq - a_pp)/(2 a_pq),
// t = sgn(theta)/(|theta| + sqrt(theta^2 + 1)), c = 1/sqrt(1 + t^2), s = t c.
// A step is one pass: the pairs split A into 2x2 blocks (rows of pair k1,
// columns of pair k2), each transformed as J_k1^T B J_k2 by one thread; the
// blocks with k1 < k2 also write their transpose, so A stays exactly
// symmetric and only the upper block triangle is computed.  V <- V J in the
// same pass.
// A (symmetrised, then destroyed) and V live in shared memory; on return w
// (shared, n) holds the eigenvalues in ascending order and V's columns the matching eigenvectors.
// scratch: shared ints/doubles of size >= 3 * RKS_NBF_CAP.  Returns the sweep
// count, or -1 when max_sweeps was exhausted before convergence.
__device__ inline int jacobi(double *A, double *V, double *w, int n, double *red, int *perm,
                             double *cs, int max_sweeps = 40) {
    const int ne = n + (n & 1);  // even count; index n is a dummy when n is odd
    const int npair = ne / 2;
    const int nblk = npair * (npair + 1) / 2;
    // the block update reads one triangle: make A exactly symmetric first
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx % n;
        V[idx] = i == j ? 1.0 : 0.0;
        if (i < j) {
            const double v = 0.5 * (A[idx] + A[j * n + i]);
            A[idx] = v;
            A[j * n + i] = v;
        }
    }
    __syncthreads();
    double *cc = cs, *ss = cs + RKS_NBF_CAP / 2 + 1;
    int *pp = perm + RKS_NBF_CAP + 2, *qq = pp + RKS_NBF_CAP / 2 + 1;
    int sweep = 0;
    for (; sweep < max_sweeps; sweep++) {
        // convergence test: off-diagonal Frobenius norm vs diagonal
        double off = 0.0, dia = 0.0;
        for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
            double a = A[i];
            if (i / n == i % n) dia += a * a; else off += a * a;
        }
        off = block_sum(off, red);
        dia = block_sum(dia, red);
        if (off <= 1e-30 * dia || off == 0.0) break;
        for (int step = 0; step < ne - 1; step++) {
            for (int k = threadIdx.x; k < npair; k += blockDim.x) {
                // index at position i after `step` rotations
                const int ik = ne - 1 - k;
                int p = k == 0 ? 0 : (k - 1 - step + 2 * (ne - 1)) % (ne - 1) + 1;
                int q = (ik - 1 - step + 2 * (ne - 1)) % (ne - 1) + 1;
                if (p > q) { int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0;
                if (q < n) {
                    double apq = A[p * n + q];
                    double app = A[p * n + p], aqq = A[q * n + q];
                    if (fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
                        double th = (aqq - app) / (2.0 * apq);
                        double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                cc[k] = c; ss[k] = s; pp[k] = p; qq[k] = q;
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < nblk + npair * n; idx += blockDim.x) {
                if (idx < nblk) {
                    // block (k1, k2), k1 <= k2, from the triangular index
                    int k2 = (int)((sqrtf(8.f * (float)idx + 1.f) - 1.f) * 0.5f);
                    while (k2 * (k2 + 1) / 2 > idx) k2--;
                    while ((k2 + 1) * (k2 + 2) / 2 <= idx) k2++;
                    const int k1 = idx - k2 * (k2 + 1) / 2;
                    const double s1 = ss[k1], s2 = ss[k2];
                    if (s1 == 0.0 && s2 == 0.0) continue;
                    const double c1 = cc[k1], c2 = cc[k2];
                    const int p1 = pp[k1], q1 = qq[k1], p2 = pp[k2], q2 = qq[k2];
                    const bool r1 = q1 < n, r2 = q2 < n;  // q is the dummy index when n is odd
                    const double bpp = A[p1 * n + p2], bpq = r2 ? A[p1 * n + q2] : 0.0;
                    const double bqp = r1 ? A[q1 * n + p2] : 0.0, bqq = r1 && r2 ? A[q1 * n + q2] : 0.0;
                    // rows of pair k1, then columns of pair k2
                    const double tpp = c1 * bpp - s1 * bqp, tpq = c1 * bpq - s1 * bqq;
                    const double tqp = s1 * bpp + c1 * bqp, tqq = s1 * bpq + c1 * bqq;
                    const double upp = c2 * tpp - s2 * tpq, upq = s2 * tpp + c2 * tpq;
                    const double uqp = c2 * tqp - s2 * tqq, uqq = s2 * tqp + c2 * tqq;
                    if (k1 == k2) {  // diagonal block: p1 = p2, q1 = q2
                        A[p1 * n + p1] = upp;
                        if (r1) {
                            A[p1 * n + q1] = upq;
                            A[q1 * n + p1] = upq;
                            A[q1 * n + q1] = uqq;
                        }
                    } else {
                        A[p1 * n + p2] = upp; A[p2 * n + p1] = upp;
                        if (r2) { A[p1 * n + q2] = upq; A[q2 * n + p1] = upq; }
                        if (r1) { A[q1 * n + p2] = uqp; A[p2 * n + q1] = uqp; }
                        if (r1 && r2) { A[q1 * n + q2] = uqq; A[q2 * n + q1] = uqq; }
                    }
                } else {
                    // columns p, q of V
                    const int j = idx - nblk, k = j / n, i = j % n;
                    const int p = pp[k], q = qq[k];
                    if (q >= n || ss[k] == 0.0) continue;
                    const double c = cc[k], s = ss[k];
                    const double vp = V[i * n + p], vq = V[i * n + q];
                    V[i * n + p] = c * vp - s * vq;
                    V[i * n + q] = s * vp + c * vq;
                }
            }
            __syncthreads();
        }
    }
    // sort ascending: rank of each eigenvalue
    double *tmpw = cs;  // reuse (n <= RKS_NBF_CAP)
    for (int i = threadIdx.x; i < n; i += blockDim.x) tmpw[i] = A[i * n + i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double wi = tmpw[i];
        int r = 0;
        for (int j = 0; j < n; j++) {
            double wj = tmpw[j];
            r += (wj < wi) || (wj == wi && j < i);
        }
        perm[i] = r;
        w[r] = wi;
    }
    __syncthreads();
    // permute V's columns into A (as scratch), then copy back
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        int i = idx / n, j = idx % n;
        A[i * n + perm[j]] = V[idx];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) V[idx] = A[idx];
    __syncthreads();
    return sweep < max_sweeps ? sweep : -1;
}

}  // namespace la
