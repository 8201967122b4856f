// Iteration-0 kernels (the paper's precompute of V, T, S and I^2e, Section
// 3.1): Boys table, quadrature tables, one-electron integrals, Schwarz
// screening and the packed two-electron store, and the molecular grid.
//
// Packing convention (the paper stores I^2e once per 8-fold symmetry orbit,
// Section 3.2 footnote; screening and order are this library's definition):
//  * shells: s shells (atom order, 1s then 2s) then p shells (atom order);
//  * candidate pairs P >= Q ordered by (l_P + l_Q, P, Q);
//  * Q_PQ = sqrt(max_{i in P, j in Q} |(ij|ij)|) in FP64; pair kept iff
//    Q_PQ Q_max >= tau; quartet (pq, rs <= pq) kept iff Q_pq Q_rs >= tau, tau = 1e-12;
//  * the store holds, row by row (pq) and within a row by rs, each kept quartet's
//    full n_P n_Q n_R n_S block, row-major (i, j, k, l).
#include "common.cuh"
#include "eri.cuh"
#include "kernels.h"

#define TAU_SCHWARZ 1e-12

// ------------------------------------------------------------ Boys table
// Row i: T_i = i h; columns F_0..F_(ncol-1), by the series
// F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)), summed in FP64.
__global__ void boys_table_kernel(double *t64, float *t32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= BOYS_N64) return;
    double T = i * BOYS_H;
    for (int m = 0; m < BOYS_COL64; m++) {
        double term = 1.0 / (2 * m + 1), sum = term;
        for (int k = 1; k < 1000; k++) {
            term *= 2.0 * T / (2 * m + 2 * k + 1);
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        double f = exp(-T) * sum;
        t64[i * BOYS_COL64 + m] = f;
        if (i < BOYS_N32 && m < BOYS_COL32) t32[i * BOYS_COL32 + m] = (float)f;
    }
}

// Evaluate F_0..F_mmax at given T (unit test entry).
template <typename T, int L>
__global__ void boys_eval_kernel(const double *Targ, double *out, int n, const T *tab) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T F[L + 1];
    boys_eval<T, L>((T)Targ[i], tab, F);
    for (int m = 0; m <= L; m++) out[i * (L + 1) + m] = (double)F[m];
}

void launch_boys_eval(int mmax, int n, const double *dT, double *dout, int fp32, const double *t64,
                      const float *t32, cudaStream_t s) {
    int g = (n + 127) / 128;
    if (fp32) {
        switch (mmax) {
        case 0: boys_eval_kernel<float, 0><<<g, 128, 0, s>>>(dT, dout, n, t32); break;
        case 1: boys_eval_kernel<float, 1><<<g, 128, 0, s>>>(dT, dout, n, t32); break;
        case 2: boys_eval_kernel<float, 2><<<g, 128, 0, s>>>(dT, dout, n, t32); break;
        case 3: boys_eval_kernel<float, 3><<<g, 128, 0, s>>>(dT, dout, n, t32); break;
        default: boys_eval_kernel<float, 4><<<g, 128, 0, s>>>(dT, dout, n, t32); break;
        }
    } else {
        switch (mmax) {
        case 0: boys_eval_kernel<double, 0><<<g, 128, 0, s>>>(dT, dout, n, t64); break;
        case 1: boys_eval_kernel<double, 1><<<g, 128, 0, s>>>(dT, dout, n, t64); break;
        case 2: boys_eval_kernel<double, 2><<<g, 128, 0, s>>>(dT, dout, n, t64); break;
        case 3: boys_eval_kernel<double, 3><<<g, 128, 0, s>>>(dT, dout, n, t64); break;
        default: boys_eval_kernel<double, 4><<<g, 128, 0, s>>>(dT, dout, n, t64); break;
        }
    }
}

void launch_boys_table(double *t64, float *t32, cudaStream_t s) {
    boys_table_kernel<<<(BOYS_N64 + 127) / 128, 128, 0, s>>>(t64, t32);
}

// ------------------------------------------------------ quadrature tables
// Radial: Treutler-Ahlrichs M4 map of Gauss-Chebyshev (2nd kind) nodes,
//   x_i = cos(i pi/(n+1)), r = (xi/ln2)(1+x)^0.6 ln(2/(1-x)),
//   w_i = pi/(n+1) sin(i pi/(n+1)) dr/dx r^2,  xi: H 0.8, C 1.1, N 0.9, O 0.9, F 0.9
//   (Treutler & Ahlrichs, J. Chem. Phys. 102, 346 (1995)).
// Angular: Gauss-Legendre nodes in cos(theta), ascending (Newton iteration on P_n), times
//   phi_k = 2 pi k / n_phi, weight w_GL 2 pi / n_phi.
// Layout: rad[(e * n_rad + i) * 2 + {0: r, 1: w}], ang[(j * n_phi + k) * 4 + {x, y, z, w}].
__global__ void quad_table_kernel(double *rad, double *ang, int n_rad, int n_theta, int n_phi) {
    const double xi_tab[5] = {0.8, 1.1, 0.9, 0.9, 0.9};
    int t = threadIdx.x;
    for (int idx = t; idx < 5 * n_rad; idx += blockDim.x) {
        int e = idx / n_rad, i = idx % n_rad + 1;
        double th = i * M_PI / (n_rad + 1);
        double x = cos(th);
        double c = xi_tab[e] / log(2.0);
        double r = c * pow(1.0 + x, 0.6) * log(2.0 / (1.0 - x));
        double drdx = c * (0.6 * pow(1.0 + x, -0.4) * log(2.0 / (1.0 - x)) + pow(1.0 + x, 0.6) / (1.0 - x));
        rad[idx * 2 + 0] = r;
        rad[idx * 2 + 1] = M_PI / (n_rad + 1) * sin(th) * drdx * r * r;
    }
    __shared__ double gl_x[64], gl_w[64];
    for (int i = t; i < n_theta; i += blockDim.x) {
        // i-th root of P_n, descending from near 1
        double z = cos(M_PI * (i + 0.75) / (n_theta + 0.5));
        double pd = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n_theta; k++) {
                double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n_theta == 1) { p1 = z; p0 = 1.0; }
            pd = n_theta * (z * p1 - p0) / (z * z - 1.0);  // P_n'
            double dz = p1 / pd;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n_theta; k++) {
                double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            pd = n_theta * (z * p1 - p0) / (z * z - 1.0);
        }
        // roots come out descending; store ascending in cos(theta)
        gl_x[n_theta - 1 - i] = z;
        gl_w[n_theta - 1 - i] = 2.0 / ((1.0 - z * z) * pd * pd);
    }
    __syncthreads();
    for (int idx = t; idx < n_theta * n_phi; idx += blockDim.x) {
        int j = idx / n_phi, k = idx % n_phi;
        double ct = gl_x[j], st = sqrt(fmax(0.0, 1.0 - ct * ct));
        double ph = 2.0 * M_PI * k / n_phi;
        ang[idx * 4 + 0] = st * cos(ph);
        ang[idx * 4 + 1] = st * sin(ph);
        ang[idx * 4 + 2] = ct;
        ang[idx * 4 + 3] = gl_w[j] * 2.0 * M_PI / n_phi;
    }
}

void launch_quad_tables(double *rad, double *ang, int n_rad, int n_theta, int n_phi, cudaStream_t s) {
    quad_table_kernel<<<1, 256, 0, s>>>(rad, ang, n_rad, n_theta, n_phi);
}

// --------------------------------------------------------- shell helpers
template <typename T>
__device__ __forceinline__ void load_shell(const DevBatch &b, int gsh, T *C, eri::Prim3<T> &p) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
        C[k] = (T)b.sh_xyz[gsh * 3 + k];
        p.e[k] = (T)b.sh_ex[gsh * 3 + k];
        p.c[k] = (T)b.sh_co[gsh * 3 + k];
    }
}

// ------------------------------------------------- one-electron integrals
// S, T and V for every candidate pair (P >= Q), FP64, Obara-Saika:
//  (s|s) = (pi/zeta)^(3/2) exp(-xi AB^2),  xi = ab/zeta;
//  (p_i|s) = PA_i (s|s); (p_i|p_j) = PA_i (s|p_j) + delta_ij/(2 zeta) (s|s);
//  (s|T|s) = xi (3 - 2 xi AB^2)(s|s);  (a+1_i|T|b) = PA_i (a|T|b)
//     + [N_i(a)(a-1_i|T|b) + N_i(b)(a|T|b-1_i)]/(2 zeta) + 2 xi [(a+1_i|b) - N_i(a)/(2a) (a-1_i|b)];
//  (s|V_C|s)^m = -Z_C 2 pi/zeta exp(-xi AB^2) F_m(zeta PC^2);
//  (a+1_i|V|b)^m = PA_i (a|V|b)^m - PC_i (a|V|b)^(m+1)
//     + N_i(a)/(2 zeta) [(a-1_i|V|b)^m - (a-1_i|V|b)^(m+1)] + N_i(b)/(2 zeta) [...].
__global__ void onee_kernel(DevBatch b, int ncand_total) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ncand_total) return;
    int m = b.cand_mol[g];
    const MolDesc md = b.mol[m];
    int2 pq = b.cand[g];
    int P = md.sh0 + pq.x, Q = md.sh0 + pq.y;
    int lP = b.sh_l[P], lQ = b.sh_l[Q];
    double A[3], B[3];
    for (int k = 0; k < 3; k++) { A[k] = b.sh_xyz[P * 3 + k]; B[k] = b.sh_xyz[Q * 3 + k]; }
    double AB2 = 0;
    for (int k = 0; k < 3; k++) AB2 += (A[k] - B[k]) * (A[k] - B[k]);
    int na = lP ? 3 : 1, nb = lQ ? 3 : 1;
    double S[9] = {0}, Tk[9] = {0}, V[9] = {0};
    for (int ia = 0; ia < 3; ia++)
        for (int ib = 0; ib < 3; ib++) {
            double a = b.sh_ex[P * 3 + ia], bb = b.sh_ex[Q * 3 + ib];
            double cc = b.sh_co[P * 3 + ia] * b.sh_co[Q * 3 + ib];
            double z = a + bb, oz = 1.0 / z, xi = a * bb * oz;
            double Pc[3], PA[3], PB[3];
            for (int k = 0; k < 3; k++) {
                Pc[k] = (a * A[k] + bb * B[k]) * oz;
                PA[k] = Pc[k] - A[k];
                PB[k] = Pc[k] - B[k];
            }
            double ex = exp(-xi * AB2);
            double s00 = pow(M_PI * oz, 1.5) * ex;
            double t00 = xi * (3.0 - 2.0 * xi * AB2) * s00;
            // overlap and kinetic
            for (int i = 0; i < na; i++)
                for (int j = 0; j < nb; j++) {
                    double s, t;
                    if (!lP && !lQ) { s = s00; t = t00; }
                    else if (lP && !lQ) { s = PA[i] * s00; t = PA[i] * t00 + 2.0 * xi * s; }
                    else if (!lP && lQ) { s = PB[j] * s00; t = PB[j] * t00 + 2.0 * xi * s; }
                    else {
                        double s_sp = PB[j] * s00;                     // (s|p_j)
                        double t_sp = PB[j] * t00 + 2.0 * xi * s_sp;   // (s|T|p_j)
                        s = PA[i] * s_sp + (i == j ? 0.5 * oz * s00 : 0.0);
                        t = PA[i] * t_sp + (i == j ? 0.5 * oz * t00 : 0.0) + 2.0 * xi * s;
                    }
                    S[i * nb + j] += cc * s;
                    Tk[i * nb + j] += cc * t;
                }
            // nuclear attraction
            for (int c = 0; c < md.natom; c++) {
                double Zc = (double)b.Z[md.atom0 + c];
                double PC[3], PC2 = 0;
                for (int k = 0; k < 3; k++) {
                    PC[k] = Pc[k] - b.axyz[(md.atom0 + c) * 3 + k];
                    PC2 += PC[k] * PC[k];
                }
                double F[3];
                boys_eval<double, 2>(z * PC2, b.boys64, F);
                double v0[3];
                for (int mm = 0; mm < 3; mm++) v0[mm] = -Zc * 2.0 * M_PI * oz * ex * F[mm];
                for (int i = 0; i < na; i++)
                    for (int j = 0; j < nb; j++) {
                        double v;
                        if (!lP && !lQ) v = v0[0];
                        else if (lP && !lQ) v = PA[i] * v0[0] - PC[i] * v0[1];
                        else if (!lP && lQ) v = PB[j] * v0[0] - PC[j] * v0[1];
                        else {
                            double sp0 = PB[j] * v0[0] - PC[j] * v0[1];  // (s|V|p_j)^0
                            double sp1 = PB[j] * v0[1] - PC[j] * v0[2];  // (s|V|p_j)^1
                            v = PA[i] * sp0 - PC[i] * sp1 + (i == j ? 0.5 * oz * (v0[0] - v0[1]) : 0.0);
                        }
                        V[i * nb + j] += cc * v;
                    }
            }
        }
    int n = md.nbf;
    double *Sm = b.mat + md.mat0 + (long long)M_S * n * n;
    double *Tm = b.mat + md.mat0 + (long long)M_T * n * n;
    double *Vm = b.mat + md.mat0 + (long long)M_V * n * n;
    int a0 = b.sh_ao0[P], b0 = b.sh_ao0[Q];
    for (int i = 0; i < na; i++)
        for (int j = 0; j < nb; j++) {
            int r = a0 + i, c = b0 + j;
            Sm[r * n + c] = S[i * nb + j]; Sm[c * n + r] = S[i * nb + j];
            Tm[r * n + c] = Tk[i * nb + j]; Tm[c * n + r] = Tk[i * nb + j];
            Vm[r * n + c] = V[i * nb + j]; Vm[c * n + r] = V[i * nb + j];
        }
}

void launch_onee(const DevBatch &b, int ncand, cudaStream_t s) {
    onee_kernel<<<(ncand + 127) / 128, 128, 0, s>>>(b, ncand);
}

// ------------------------------------------------------------- Schwarz
template <int L1, int L2>
__device__ double schwarz_diag(const DevBatch &b, int P, int Q) {
    double A[3], B[3];
    eri::Prim3<double> pa, pb;
    load_shell<double>(b, P, A, pa);
    load_shell<double>(b, Q, B, pb);
    constexpr int N = (L1 ? 3 : 1) * (L2 ? 3 : 1);
    double out[N * N];
    eri::quartet<double, L1, L2, L1, L2>(A, B, A, B, pa, pb, pa, pb, b.boys64, out);
    double mx = 0.0;
#pragma unroll
    for (int x = 0; x < N; x++) mx = fmax(mx, fabs(out[x * N + x]));
    return sqrt(mx);
}

__global__ void schwarz_kernel(DevBatch b, int ncand_total) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ncand_total) return;
    int m = b.cand_mol[g];
    const MolDesc md = b.mol[m];
    int2 pq = b.cand[g];
    int P = md.sh0 + pq.x, Q = md.sh0 + pq.y;
    int c = b.sh_l[P] * 2 + b.sh_l[Q];
    double q;
    if (c == 0) q = schwarz_diag<0, 0>(b, P, Q);
    else if (c == 2) q = schwarz_diag<1, 0>(b, P, Q);
    else q = schwarz_diag<1, 1>(b, P, Q);
    b.cand_q[g] = q;
}

void launch_schwarz(const DevBatch &b, int ncand, cudaStream_t s) {
    schwarz_kernel<<<(ncand + 127) / 128, 128, 0, s>>>(b, ncand);
}

// ---------------------------------------------------- pair compaction
// One warp per molecule: Q_max, then a stable compaction of the candidates
// with Q_PQ Q_max >= tau.
__global__ void compact_pairs_kernel(DevBatch b) {
    int m = blockIdx.x;
    if (m >= b.nmol) return;
    const MolDesc md = b.mol[m];
    int lane = threadIdx.x;
    double qmax = 0.0;
    for (int i = lane; i < md.npair_all; i += 32) qmax = fmax(qmax, b.cand_q[md.pair0 + i]);
    for (int o = 16; o > 0; o >>= 1) qmax = fmax(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
    int cnt = 0;
    for (int i0 = 0; i0 < md.npair_all; i0 += 32) {
        int i = i0 + lane;
        bool keep = false;
        double q = 0.0;
        if (i < md.npair_all) {
            q = b.cand_q[md.pair0 + i];
            keep = q * qmax >= TAU_SCHWARZ;
        }
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            int pos = cnt + __popc(bal & ((1u << lane) - 1u));
            b.kpair[md.pair0 + pos] = b.cand[md.pair0 + i];
            b.kq[md.pair0 + pos] = q;
        }
        cnt += __popc(bal);
    }
    if (lane == 0) b.npair[m] = cnt;
}

void launch_compact_pairs(const DevBatch &b, cudaStream_t s) {
    compact_pairs_kernel<<<b.nmol, 32, 0, s>>>(b);
}

// ----------------------------------------- quartet counting per row
__device__ __forceinline__ int ncomp_l(int l) { return l ? 3 : 1; }

// Warp per (molecule, kept row r).  Writes the row's element count to
// row_off[pair0 + m + r + 1] (scanned later) and its quartet count.
__global__ void row_count_kernel(DevBatch b, int ncand_total) {
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= ncand_total) return;
    int m = b.cand_mol[w];
    const MolDesc md = b.mol[m];
    int r = w - md.pair0;
    if (r >= b.npair[m]) return;
    int2 pq = b.kpair[md.pair0 + r];
    double qpq = b.kq[md.pair0 + r];
    int npq = ncomp_l(b.sh_l[md.sh0 + pq.x]) * ncomp_l(b.sh_l[md.sh0 + pq.y]);
    long long elems = 0;
    int nq = 0, ties = 0;
    for (int s0 = 0; s0 <= r; s0 += 32) {
        int s = s0 + lane;
        if (s <= r) {
            double prod = qpq * b.kq[md.pair0 + s];
            if (prod >= TAU_SCHWARZ) {
                int2 rs = b.kpair[md.pair0 + s];
                elems += npq * ncomp_l(b.sh_l[md.sh0 + rs.x]) * ncomp_l(b.sh_l[md.sh0 + rs.y]);
                nq++;
            }
            if (fabs(prod / TAU_SCHWARZ - 1.0) < 1e-10) ties++;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        elems += __shfl_xor_sync(0xffffffffu, elems, o);
        nq += __shfl_xor_sync(0xffffffffu, nq, o);
        ties += __shfl_xor_sync(0xffffffffu, ties, o);
    }
    if (lane == 0) {
        b.row_off[md.pair0 + m + r + 1] = elems;
        b.row_nq[md.pair0 + r] = nq;
        if (ties) atomicAdd(&b.st[m].near_ties, ties);
    }
}

void launch_row_count(const DevBatch &b, int ncand, cudaStream_t s) {
    long long threads = (long long)ncand * 32;
    row_count_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(b, ncand);
}

// One block per molecule: in-place inclusive scan of the row counts
// (row_off[base + 1 .. base + npair]) with row_off[base] = 0.
__global__ void row_scan_kernel(DevBatch b) {
    int m = blockIdx.x;
    const MolDesc md = b.mol[m];
    long long *ro = b.row_off + md.pair0 + m;
    int n = b.npair[m];
    __shared__ long long carry;
    __shared__ long long wsum[32];
    __shared__ int nqs[32];
    if (threadIdx.x == 0) { carry = 0; ro[0] = 0; }
    int nq_tot = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        int i = base + threadIdx.x;
        long long v = (i < n) ? ro[i + 1] : 0;
        int q = (i < n) ? b.row_nq[md.pair0 + i] : 0;
        nq_tot += q;
        // block inclusive scan
        int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int nw = blockDim.x >> 5;
            long long t = (lane < nw) ? wsum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                long long y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < nw) wsum[lane] = t;
        }
        __syncthreads();
        long long pre = (wid > 0 ? wsum[wid - 1] : 0) + carry;
        if (i < n) ro[i + 1] = x + pre;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = x + pre;
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) nq_tot += __shfl_xor_sync(0xffffffffu, nq_tot, o);
    if ((threadIdx.x & 31) == 0) nqs[threadIdx.x >> 5] = nq_tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += nqs[i];
        b.st[m].n_quartets = t;
        b.st[m].n_elem = ro[n];
        if (ro[n] > md.eri_cap) b.st[m].err_flag |= 1;  // cannot happen: capacity is the unscreened bound
    }
}

void launch_row_scan(const DevBatch &b, cudaStream_t s) { row_scan_kernel<<<b.nmol, 256, 0, s>>>(b); }

// ------------------------------------------------------ primitive pairs
// For every kept pair (P, Q) and primitive pair (a, b), in FP64:
//   K = c_a c_b exp(-ab/(a+b) |A-B|^2), zeta = a + b, P - A = b (B - A)/zeta,
// stored in the ERI precision.  The FP32 ERI path then never forms an
// exponent or a Boys argument from rounded absolute coordinates.
template <typename T>
__global__ void pair_prim_kernel(DevBatch b, int ncand_total, void *dst) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ncand_total) return;
    int m = b.cand_mol[g];
    const MolDesc md = b.mol[m];
    int r = g - md.pair0;
    if (r >= b.npair[m]) return;
    int2 pq = b.kpair[md.pair0 + r];
    int P = md.sh0 + pq.x, Q = md.sh0 + pq.y;
    double AB[3], ab2 = 0;
    for (int k = 0; k < 3; k++) {
        AB[k] = b.sh_xyz[P * 3 + k] - b.sh_xyz[Q * 3 + k];
        ab2 += AB[k] * AB[k];
    }
    eri::PrimPair<T> *out = (eri::PrimPair<T> *)dst + (long long)(md.pair0 + r) * (RKS_MAXP * RKS_MAXP);
    for (int ia = 0; ia < RKS_MAXP; ia++)
        for (int ib = 0; ib < RKS_MAXP; ib++) {
            const double a = b.sh_ex[P * 3 + ia], bb = b.sh_ex[Q * 3 + ib];
            const double z = a + bb;
            eri::PrimPair<T> pp;
            pp.K = (T)(b.sh_co[P * 3 + ia] * b.sh_co[Q * 3 + ib] * exp(-a * bb / z * ab2));
            pp.z = (T)z;
            pp.px = (T)(-bb / z * AB[0]);
            pp.py = (T)(-bb / z * AB[1]);
            pp.pz = (T)(-bb / z * AB[2]);
            out[ia * RKS_MAXP + ib] = pp;
        }
}

void launch_pair_prim(const DevBatch &b, int ncand, int fp32, cudaStream_t s) {
    if (fp32) {
        pair_prim_kernel<float><<<(ncand + 127) / 128, 128, 0, s>>>(b, ncand, b.pairprim);
        if (b.pairprim64) pair_prim_kernel<double><<<(ncand + 127) / 128, 128, 0, s>>>(b, ncand, b.pairprim64);
    } else {
        pair_prim_kernel<double><<<(ncand + 127) / 128, 128, 0, s>>>(b, ncand, b.pairprim);
    }
}

// ------------------------------------------------------------ ERI store
template <typename T, int LA, int LB, int LC, int LD>
__device__ __forceinline__ void quartet_to_store(const DevBatch &b, const MolDesc &md, int r, int s, int P, int Q,
                                                 int R, int S, const T *tab, T *dst) {
    T AB[3], CD[3], AC[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        AB[k] = (T)(b.sh_xyz[P * 3 + k] - b.sh_xyz[Q * 3 + k]);
        CD[k] = (T)(b.sh_xyz[R * 3 + k] - b.sh_xyz[S * 3 + k]);
        AC[k] = (T)(b.sh_xyz[P * 3 + k] - b.sh_xyz[R * 3 + k]);
    }
    const eri::PrimPair<T> *pp = (const eri::PrimPair<T> *)b.pairprim;
    constexpr int N = (LA ? 3 : 1) * (LB ? 3 : 1) * (LC ? 3 : 1) * (LD ? 3 : 1);
    T out[N];
    eri::quartet_pd<T, LA, LB, LC, LD>(pp + (long long)(md.pair0 + r) * 9, pp + (long long)(md.pair0 + s) * 9, AB,
                                       CD, AC, tab, out);
#pragma unroll
    for (int x = 0; x < N; x++) dst[x] = out[x];
}

// Warp per (molecule, kept row pq): lanes take rs = 0..pq in chunks of 32,
// screen, take offsets from a warp prefix sum and write their blocks.
template <typename T>
__global__ void eri_store_kernel(DevBatch b, int ncand_total) {
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= ncand_total) return;
    int m = b.cand_mol[w];
    const MolDesc md = b.mol[m];
    int r = w - md.pair0;
    if (r >= b.npair[m]) return;
    const T *tab = nullptr;
    if constexpr (sizeof(T) == 8) tab = (const T *)b.boys64; else tab = (const T *)b.boys32;
    T *store = (T *)b.store + md.eri0;
    int2 pq = b.kpair[md.pair0 + r];
    double qpq = b.kq[md.pair0 + r];
    int P = md.sh0 + pq.x, Q = md.sh0 + pq.y;
    int lP = b.sh_l[P], lQ = b.sh_l[Q];
    int npq = ncomp_l(lP) * ncomp_l(lQ);
    long long base = b.row_off[md.pair0 + m + r];
    for (int s0 = 0; s0 <= r; s0 += 32) {
        int s = s0 + lane;
        bool keep = false;
        int R = 0, S = 0, nel = 0;
        if (s <= r && qpq * b.kq[md.pair0 + s] >= TAU_SCHWARZ) {
            int2 rs = b.kpair[md.pair0 + s];
            R = md.sh0 + rs.x;
            S = md.sh0 + rs.y;
            keep = true;
            nel = npq * ncomp_l(b.sh_l[R]) * ncomp_l(b.sh_l[S]);
        }
        int x = nel;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        int tot = __shfl_sync(0xffffffffu, x, 31);
        long long off = base + x - nel;
        if (keep) {
            T *dst = store + off;
            int lR = b.sh_l[R], lS = b.sh_l[S];
            int cls = (lP << 3) | (lQ << 2) | (lR << 1) | lS;
            switch (cls) {
            case 0x0: quartet_to_store<T, 0, 0, 0, 0>(b, md, r, s, P, Q, R, S, tab, dst); break;
            case 0x8: quartet_to_store<T, 1, 0, 0, 0>(b, md, r, s, P, Q, R, S, tab, dst); break;
            case 0xA: quartet_to_store<T, 1, 0, 1, 0>(b, md, r, s, P, Q, R, S, tab, dst); break;
            case 0xC: quartet_to_store<T, 1, 1, 0, 0>(b, md, r, s, P, Q, R, S, tab, dst); break;
            case 0xE: quartet_to_store<T, 1, 1, 1, 0>(b, md, r, s, P, Q, R, S, tab, dst); break;
            case 0xF: quartet_to_store<T, 1, 1, 1, 1>(b, md, r, s, P, Q, R, S, tab, dst); break;
            default: atomicOr(&b.st[m].err_flag, 2); break;  // class outside the packing order
            }
        }
        base += tot;
    }
}

void launch_eri_store(const DevBatch &b, int ncand, int fp32, cudaStream_t s) {
    long long threads = (long long)ncand * 32;
    unsigned g = (unsigned)((threads + 127) / 128);
    if (fp32) eri_store_kernel<float><<<g, 128, 0, s>>>(b, ncand);
    else eri_store_kernel<double><<<g, 128, 0, s>>>(b, ncand);
}

// ------------------------------------------------------------------ grid
// Thread per grid point (blocks of 128 belong to one molecule).  Point p of a
// molecule: atom A = p / (n_rad n_ang), then radial index, then angular index.
// Points are stored as offsets r * u from their own nucleus (A is implied by
// the index), so every point-to-centre vector is formed as
// (R_A - R_B) [from FP64 coordinates] + offset and keeps full relative
// precision near nuclei even in FP32.
// Becke partition (A. D. Becke, J. Chem. Phys. 88, 2547 (1988)):
//   mu_BC = (|r - R_B| - |r - R_C|)/|R_B - R_C|, f = p(p(p(mu))), p(x) = 1.5x - 0.5x^3,
//   s = (1 - f)/2, P_B = prod_{C != B} s(mu_BC), w = w_rad w_ang P_A / sum_B P_B.
template <typename T>
__global__ void grid_build_kernel(DevBatch b, const int *blk_mol, const double *rad, const double *ang) {
    extern __shared__ unsigned char smem_raw[];
    long long blk = blockIdx.x;
    int m = blk_mol[blk];
    const MolDesc md = b.mol[m];
    const int nat = md.natom;
    T *invR = (T *)smem_raw;            // [nat][nat]
    const double *ax = b.axyz + md.atom0 * 3;
    for (int i = threadIdx.x; i < nat * nat; i += blockDim.x) {
        int B = i / nat, C = i % nat;
        double dx = ax[B * 3] - ax[C * 3], dy = ax[B * 3 + 1] - ax[C * 3 + 1], dz = ax[B * 3 + 2] - ax[C * 3 + 2];
        invR[i] = (B == C) ? (T)0 : (T)(1.0 / sqrt(dx * dx + dy * dy + dz * dz));
    }
    __syncthreads();
    long long gp = blk * RKS_PTS_BLOCK + threadIdx.x;  // global point index
    long long lp = gp - md.pts0;                       // local
    T *gx = (T *)b.gx, *gy = (T *)b.gy, *gz = (T *)b.gz, *gw = (T *)b.gw;
    const int nang = b.n_theta * b.n_phi;
    const int npa = b.n_rad * nang;
    if (lp >= md.npts) {  // padding: weight 0 at the last nucleus (owner index clamps there)
        gx[gp] = (T)0; gy[gp] = (T)0; gz[gp] = (T)0; gw[gp] = (T)0;
        return;
    }
    int A = (int)(lp / npa);
    int rem = (int)(lp % npa);
    int ir = rem / nang, ia = rem % nang;
    int z = b.Z[md.atom0 + A];
    int e = z == 1 ? 0 : (z == 6 ? 1 : (z == 7 ? 2 : (z == 8 ? 3 : 4)));
    double r = rad[(e * b.n_rad + ir) * 2 + 0], wr = rad[(e * b.n_rad + ir) * 2 + 1];
    double dxn = ang[ia * 4 + 0], dyn = ang[ia * 4 + 1], dzn = ang[ia * 4 + 2], wa = ang[ia * 4 + 3];
    const T ox = (T)(r * dxn), oy = (T)(r * dyn), oz = (T)(r * dzn);
    // distances to every nucleus (local array)
    T dist[128];
    for (int B = 0; B < nat; B++) {
        T dx = (T)(ax[A * 3] - ax[B * 3]) + ox, dy = (T)(ax[A * 3 + 1] - ax[B * 3 + 1]) + oy;
        T dz = (T)(ax[A * 3 + 2] - ax[B * 3 + 2]) + oz;
        dist[B] = dev_sqrt(dx * dx + dy * dy + dz * dz);
    }
    // each unordered pair once: mu_CB = -mu_BC and the iterated p is odd, so
    // s(mu_CB) = (1 + f_BC) / 2 while s(mu_BC) = (1 - f_BC) / 2
    T P[128];
    for (int B = 0; B < nat; B++) P[B] = (T)1;
    for (int B = 0; B < nat; B++) {
        T PB = P[B];
        for (int C = B + 1; C < nat; C++) {
            T mu = (dist[B] - dist[C]) * invR[B * nat + C];
            T f = mu;
            for (int it = 0; it < b.becke_iters; it++) f = (T)1.5 * f - (T)0.5 * f * f * f;
            PB *= (T)0.5 * ((T)1 - f);
            P[C] *= (T)0.5 * ((T)1 + f);
        }
        P[B] = PB;
    }
    T sumP = 0;
    for (int B = 0; B < nat; B++) sumP += P[B];
    const T PA = P[A];
    gx[gp] = ox; gy[gp] = oy; gz[gp] = oz;
    gw[gp] = (T)(wr * wa) * PA / sumP;
}

int launch_grid_build(const DevBatch &b, long long nblk_total, const int *blk_mol, const double *rad,
                      const double *ang, int max_atoms, cudaStream_t s) {
    size_t sm = (size_t)(max_atoms * max_atoms) * (b.precision ? sizeof(float) : sizeof(double));
    if (b.precision) {
        cudaFuncSetAttribute(grid_build_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        grid_build_kernel<float><<<(unsigned)nblk_total, RKS_PTS_BLOCK, sm, s>>>(b, blk_mol, rad, ang);
    } else {
        cudaFuncSetAttribute(grid_build_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        grid_build_kernel<double><<<(unsigned)nblk_total, RKS_PTS_BLOCK, sm, s>>>(b, blk_mol, rad, ang);
    }
    return 0;
}
