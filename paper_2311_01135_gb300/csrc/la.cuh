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
// rotations at once (rows, then columns), a sweep has n-1 steps.
// Rotation per pair (p, q) (Rutishauser's form): theta = (a_qq - a_pp)/(2 a_pq),
// t = sgn(theta)/(|theta| + sqrt(theta^2 + 1)), c = 1/sqrt(1 + t^2), s = t c.
// A (destroyed) and V live in shared memory; on return w (shared, n) holds the
// eigenvalues in ascending order and V's columns the matching eigenvectors.
// scratch: shared ints/doubles of size >= 3 * RKS_NBF_CAP.  Returns the sweep
// count, or -1 when max_sweeps was exhausted before convergence.
__device__ inline int jacobi(double *A, double *V, double *w, int n, double *red, int *perm,
                             double *cs, int max_sweeps = 40) {
    const int ne = n + (n & 1);  // even count; index n is a dummy when n is odd
    const int npair = ne / 2;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) V[i] = (i / n == i % n) ? 1.0 : 0.0;
    for (int i = threadIdx.x; i < ne; i += blockDim.x) perm[i] = i;
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
                int p = perm[k], q = perm[ne - 1 - k];
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
            // rows: row_p <- c row_p - s row_q; row_q <- s row_p + c row_q
            for (int idx = threadIdx.x; idx < npair * n; idx += blockDim.x) {
                int k = idx / n, j = idx % n;
                int p = pp[k], q = qq[k];
                if (q >= n || ss[k] == 0.0) continue;
                double c = cc[k], s = ss[k];
                double ap = A[p * n + j], aq = A[q * n + j];
                A[p * n + j] = c * ap - s * aq;
                A[q * n + j] = s * ap + c * aq;
            }
            __syncthreads();
            // columns of A and V
            for (int idx = threadIdx.x; idx < npair * n; idx += blockDim.x) {
                int k = idx / n, i = idx % n;
                int p = pp[k], q = qq[k];
                if (q >= n || ss[k] == 0.0) continue;
                double c = cc[k], s = ss[k];
                double ap = A[i * n + p], aq = A[i * n + q];
                A[i * n + p] = c * ap - s * aq;
                A[i * n + q] = s * ap + c * aq;
                double vp = V[i * n + p], vq = V[i * n + q];
                V[i * n + p] = c * vp - s * vq;
                V[i * n + q] = s * vp + c * vq;
            }
            __syncthreads();
            // rotate positions 1..ne-1
            if (threadIdx.x == 0) {
                int last = perm[ne - 1];
                for (int i = ne - 1; i > 1; i--) perm[i] = perm[i - 1];
                perm[1] = last;
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
