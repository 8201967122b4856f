// Two-electron repulsion integrals over contracted s/p shells on the device:
// Obara-Saika vertical recursion (VRR) per primitive quartet, contraction, then
// the Head-Gordon-Pople horizontal recursion (HRR) once per contracted quartet.
//
// This is the I^2e of the paper's iteration 0 (Section 3.1, Eq. 1) in
// chemists' notation (ab|cd) = int a(1) b(1) r12^-1 c(2) d(2); the paper's
// IPU code evaluates the same quantity with Rys quadrature (Section 3.2,
// "Libcint").  With l <= 1 per shell, the VRR builds [e0|f0] for e <= l_a + l_b,
// f <= l_c + l_d <= 2 (Cartesian s, p, d), the contraction sums over the 3x3x3x3
// primitives, and the HRR transfers angular momentum to the second centre of
// each pair:  (a, b+1_j| = (a+1_j, b| + (A - B)_j (a, b|.
//
// VRR (Obara & Saika, J. Chem. Phys. 84, 3963 (1986); Head-Gordon & Pople,
// J. Chem. Phys. 89, 5777 (1988)), zeta = a + b, eta = c + d,
// rho = zeta eta / (zeta + eta), W = (zeta P + eta Q)/(zeta + eta):
//  [e+1_i|f]^m = PA_i [e|f]^m + WP_i [e|f]^(m+1)
//              + N_i(e)/(2 zeta) ([e-1_i|f]^m - rho/zeta [e-1_i|f]^(m+1))
//              + N_i(f)/(2(zeta+eta)) [e|f-1_i]^(m+1)
//  and the mirror image on the ket with QC, WQ, eta;
//  [0|0]^m = 2 pi^(5/2) / (zeta eta sqrt(zeta+eta)) K_AB K_CD F_m(rho |PQ|^2).
//
// Cartesian component indices used throughout: 0 = s; 1..3 = p_x, p_y, p_z;
// 4..9 = d_xx, d_xy, d_xz, d_yy, d_yz, d_zz.
#pragma once
#include "boys.cuh"

namespace eri {

__host__ __device__ constexpr int DI(int c) { return c == 4 ? 0 : c == 5 ? 0 : c == 6 ? 0 : c == 7 ? 1 : c == 8 ? 1 : 2; }
__host__ __device__ constexpr int DJ(int c) { return c == 4 ? 0 : c == 5 ? 1 : c == 6 ? 2 : c == 7 ? 1 : c == 8 ? 2 : 2; }
// d component index for directions i, j
__host__ __device__ constexpr int dcomp(int i, int j) {
    return (i > j) ? dcomp(j, i) : (i == 0 ? 4 + j : (i == 1 ? 6 + j : 9));
}
// first and one-past-last component index of shell l
__host__ __device__ constexpr int cfirst(int l) { return l == 0 ? 0 : (l == 1 ? 1 : 4); }
__host__ __device__ constexpr int clast(int l) { return l == 0 ? 1 : (l == 1 ? 4 : 10); }
// N_k(c): exponent of direction k in component c
__host__ __device__ constexpr int Nk(int c, int k) {
    return c == 0 ? 0 : (c < 4 ? (c - 1 == k ? 1 : 0) : ((DI(c) == k ? 1 : 0) + (DJ(c) == k ? 1 : 0)));
}
// component index of c - 1_k (only meaningful when Nk(c, k) > 0)
__host__ __device__ constexpr int em1(int c, int k) {
    return c < 4 ? 0 : (DI(c) == k ? 1 + DJ(c) : 1 + DI(c));
}

template <typename T> struct Prim3 {
    T e[RKS_MAXP], c[RKS_MAXP];
};

// One primitive pair of a shell pair: K = c_a c_b exp(-ab/(a+b) |A-B|^2),
// zeta = a + b and P - A with P = (a A + b B)/zeta.
template <typename T> struct PrimPair {
    T K, z, px, py, pz;
};

// One contracted block (PQ|RS); A..D are the centres, the Prim3 hold exponents
// and normalised contraction coefficients.  out is row-major
// [nA][nB][nC][nD] with n = 1 (s) or 3 (p: x, y, z).
template <typename T, int LA, int LB, int LC, int LD>
__host__ __device__ __forceinline__ void quartet(const T *A, const T *B, const T *C, const T *D,
                                        const Prim3<T> &pa, const Prim3<T> &pb,
                                        const Prim3<T> &pc, const Prim3<T> &pd,
                                        const T *__restrict__ boys_tab, T *out) {
    constexpr int EM = LA + LB, FM = LC + LD, L = EM + FM;
    constexpr int E0 = cfirst(LA), E1 = clast(EM);  // e components accumulated
    constexpr int F0 = cfirst(LC), F1 = clast(FM);
    T acc[10][10];
#pragma unroll
    for (int e = E0; e < E1; e++)
#pragma unroll
        for (int f = F0; f < F1; f++) acc[e][f] = (T)0;

    T AB[3], CD[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        AB[k] = A[k] - B[k];
        CD[k] = C[k] - D[k];
    }
    const T rab2 = AB[0] * AB[0] + AB[1] * AB[1] + AB[2] * AB[2];
    const T rcd2 = CD[0] * CD[0] + CD[1] * CD[1] + CD[2] * CD[2];

#pragma unroll 1
    for (int ia = 0; ia < RKS_MAXP; ia++) {
#pragma unroll 1
        for (int ib = 0; ib < RKS_MAXP; ib++) {
            const T a = pa.e[ia], bb = pb.e[ib];
            const T zeta = a + bb, oz = (T)1 / zeta;
            const T Kab = dev_exp(-a * bb * oz * rab2) * pa.c[ia] * pb.c[ib];
            T P[3], PA[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                P[k] = (a * A[k] + bb * B[k]) * oz;
                PA[k] = P[k] - A[k];
            }
#pragma unroll 1
            for (int ic = 0; ic < RKS_MAXP; ic++) {
#pragma unroll 1
                for (int id = 0; id < RKS_MAXP; id++) {
                    const T c = pc.e[ic], d = pd.e[id];
                    const T eta = c + d, oe = (T)1 / eta;
                    const T Kcd = dev_exp(-c * d * oe * rcd2) * pc.c[ic] * pd.c[id];
                    const T ozpe = (T)1 / (zeta + eta);
                    const T rho = zeta * eta * ozpe;
                    T Q[3], QC[3], WP[3], WQ[3], PQ2 = 0;
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        Q[k] = (c * C[k] + d * D[k]) * oe;
                        QC[k] = Q[k] - C[k];
                        const T W = (zeta * P[k] + eta * Q[k]) * ozpe;
                        WP[k] = W - P[k];
                        WQ[k] = W - Q[k];
                        PQ2 += (P[k] - Q[k]) * (P[k] - Q[k]);
                    }
                    // 2 pi^(5/2) = 34.986836655249725
                    const T pref = (T)34.986836655249725 * oz * oe * dev_sqrt(ozpe) * Kab * Kcd;
                    T F[L + 1];
                    boys_eval<T, L>(rho * PQ2, boys_tab, F);
                    // ---- bra VRR: [e|s]^m for e up to EM
                    T vs[L + 1];
#pragma unroll
                    for (int m = 0; m <= L; m++) vs[m] = pref * F[m];
                    T vp[L > 0 ? L : 1][3];
                    T vd[L > 1 ? L - 1 : 1][6];
                    if constexpr (EM >= 1) {
#pragma unroll
                        for (int m = 0; m < L; m++)
#pragma unroll
                            for (int i = 0; i < 3; i++) vp[m][i] = PA[i] * vs[m] + WP[i] * vs[m + 1];
                    }
                    const T oo2z = (T)0.5 * oz, rz = rho * oz;
                    if constexpr (EM >= 2) {
#pragma unroll
                        for (int m = 0; m + 1 < L; m++)
#pragma unroll
                            for (int c6 = 0; c6 < 6; c6++) {
                                const int i = DI(c6 + 4), j = DJ(c6 + 4);
                                T v = PA[i] * vp[m][j] + WP[i] * vp[m + 1][j];
                                if (i == j) v += oo2z * (vs[m] - rz * vs[m + 1]);
                                vd[m][c6] = v;
                            }
                    }
                    // [e|s]^m accessor by component index
                    auto es = [&](int m, int e) -> T {
                        return e == 0 ? vs[m] : (e < 4 ? vp[m][e - 1] : vd[m][e - 4]);
                    };
                    if constexpr (FM == 0) {
#pragma unroll
                        for (int e = E0; e < E1; e++) acc[e][0] += es(0, e);
                    } else {
                        const T oo2ze = (T)0.5 * ozpe;
                        // [e|p_k]^m for m < FM, e from max(0, cfirst(LA) shell - 1 level)
                        constexpr int EP0 = (FM >= 2) ? cfirst(LA > 0 ? LA - 1 : 0) : E0;
                        T ep[FM][10][3];
#pragma unroll
                        for (int m = 0; m < FM; m++)
#pragma unroll
                            for (int e = EP0; e < E1; e++)
#pragma unroll
                                for (int k = 0; k < 3; k++) {
                                    T v = QC[k] * es(m, e) + WQ[k] * es(m + 1, e);
                                    if (Nk(e, k) > 0) v += (T)Nk(e, k) * oo2ze * es(m + 1, em1(e, k));
                                    ep[m][e][k] = v;
                                }
                        if constexpr (LC == 1) {
#pragma unroll
                            for (int e = E0; e < E1; e++)
#pragma unroll
                                for (int k = 0; k < 3; k++) acc[e][1 + k] += ep[0][e][k];
                        }
                        if constexpr (FM == 2) {
                            const T oo2e = (T)0.5 * oe, re = rho * oe;
#pragma unroll
                            for (int e = E0; e < E1; e++)
#pragma unroll
                                for (int c6 = 0; c6 < 6; c6++) {
                                    const int k = DI(c6 + 4), l = DJ(c6 + 4);
                                    T v = QC[k] * ep[0][e][l] + WQ[k] * ep[1][e][l];
                                    if (k == l) v += oo2e * (es(0, e) - re * es(1, e));
                                    if (Nk(e, k) > 0) v += (T)Nk(e, k) * oo2ze * ep[1][em1(e, k)][l];
                                    acc[e][4 + c6] += v;
                                }
                        }
                    }
                }
            }
        }
    }
    // ---- HRR on the ket: |c d) from |f]
    constexpr int NA = LA ? 3 : 1, NB = LB ? 3 : 1, NC = LC ? 3 : 1, ND = LD ? 3 : 1;
    T kt[10][NC * ND];
#pragma unroll
    for (int e = E0; e < E1; e++) {
        if constexpr (LD == 0) {
#pragma unroll
            for (int ic = 0; ic < NC; ic++) kt[e][ic] = acc[e][LC ? 1 + ic : 0];
        } else {  // LC = LD = 1
#pragma unroll
            for (int k = 0; k < 3; k++)
#pragma unroll
                for (int l = 0; l < 3; l++) kt[e][k * 3 + l] = acc[e][dcomp(k, l)] + CD[l] * acc[e][1 + k];
        }
    }
    // ---- HRR on the bra and store
#pragma unroll
    for (int x = 0; x < NC * ND; x++) {
        if constexpr (LB == 0) {
#pragma unroll
            for (int i = 0; i < NA; i++) out[i * NC * ND + x] = kt[LA ? 1 + i : 0][x];
        } else {
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++)
                    out[(i * 3 + j) * NC * ND + x] = kt[dcomp(i, j)][x] + AB[j] * kt[1 + i][x];
        }
    }
}

// The same block from precomputed primitive-pair data (PrimPair, formed in
// FP64 once per shell pair): K = c_a c_b exp(-ab/zeta |AB|^2), zeta and P - A.
// The centre differences AB, CD and AC are passed in (formed in FP64), so
// P - Q = AC + (P - A) - (Q - C) never cancels large coordinates; with these
// inputs an FP32 evaluation loses only rounding in the recursion itself.
template <typename T, int LA, int LB, int LC, int LD>
__host__ __device__ __forceinline__ void quartet_pd(const PrimPair<T> *__restrict__ bra,
                                                   const PrimPair<T> *__restrict__ ket, const T *AB,
                                                   const T *CD, const T *AC,
                                                   const T *__restrict__ boys_tab, T *out) {
    constexpr int EM = LA + LB, FM = LC + LD, L = EM + FM;
    constexpr int E0 = cfirst(LA), E1 = clast(EM);  // e components accumulated
    constexpr int F0 = cfirst(LC), F1 = clast(FM);
    T acc[10][10];
#pragma unroll
    for (int e = E0; e < E1; e++)
#pragma unroll
        for (int f = F0; f < F1; f++) acc[e][f] = (T)0;

#pragma unroll 1
    for (int ip = 0; ip < RKS_MAXP * RKS_MAXP; ip++) {
        {
            const T zeta = bra[ip].z, oz = (T)1 / zeta;
            const T Kab = bra[ip].K;
            T PA[3] = {bra[ip].px, bra[ip].py, bra[ip].pz};
#pragma unroll 1
            for (int iq = 0; iq < RKS_MAXP * RKS_MAXP; iq++) {
                {
                    const T eta = ket[iq].z, oe = (T)1 / eta;
                    const T Kcd = ket[iq].K;
                    const T ozpe = (T)1 / (zeta + eta);
                    const T rho = zeta * eta * ozpe;
                    T QC[3] = {ket[iq].px, ket[iq].py, ket[iq].pz};
                    T WP[3], WQ[3], PQ2 = 0;
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        const T pq = AC[k] + PA[k] - QC[k];  // P - Q
                        WP[k] = -eta * ozpe * pq;           // W - P
                        WQ[k] = zeta * ozpe * pq;           // W - Q
                        PQ2 += pq * pq;
                    }
                    // 2 pi^(5/2) = 34.986836655249725
                    const T pref = (T)34.986836655249725 * oz * oe * dev_sqrt(ozpe) * Kab * Kcd;
                    T F[L + 1];
                    boys_eval<T, L>(rho * PQ2, boys_tab, F);
                    // ---- bra VRR: [e|s]^m for e up to EM
                    T vs[L + 1];
#pragma unroll
                    for (int m = 0; m <= L; m++) vs[m] = pref * F[m];
                    T vp[L > 0 ? L : 1][3];
                    T vd[L > 1 ? L - 1 : 1][6];
                    if constexpr (EM >= 1) {
#pragma unroll
                        for (int m = 0; m < L; m++)
#pragma unroll
                            for (int i = 0; i < 3; i++) vp[m][i] = PA[i] * vs[m] + WP[i] * vs[m + 1];
                    }
                    const T oo2z = (T)0.5 * oz, rz = rho * oz;
                    if constexpr (EM >= 2) {
#pragma unroll
                        for (int m = 0; m + 1 < L; m++)
#pragma unroll
                            for (int c6 = 0; c6 < 6; c6++) {
                                const int i = DI(c6 + 4), j = DJ(c6 + 4);
                                T v = PA[i] * vp[m][j] + WP[i] * vp[m + 1][j];
                                if (i == j) v += oo2z * (vs[m] - rz * vs[m + 1]);
                                vd[m][c6] = v;
                            }
                    }
                    // [e|s]^m accessor by component index
                    auto es = [&](int m, int e) -> T {
                        return e == 0 ? vs[m] : (e < 4 ? vp[m][e - 1] : vd[m][e - 4]);
                    };
                    if constexpr (FM == 0) {
#pragma unroll
                        for (int e = E0; e < E1; e++) acc[e][0] += es(0, e);
                    } else {
                        const T oo2ze = (T)0.5 * ozpe;
                        // [e|p_k]^m for m < FM, e from max(0, cfirst(LA) shell - 1 level)
                        constexpr int EP0 = (FM >= 2) ? cfirst(LA > 0 ? LA - 1 : 0) : E0;
                        T ep[FM][10][3];
#pragma unroll
                        for (int m = 0; m < FM; m++)
#pragma unroll
                            for (int e = EP0; e < E1; e++)
#pragma unroll
                                for (int k = 0; k < 3; k++) {
                                    T v = QC[k] * es(m, e) + WQ[k] * es(m + 1, e);
                                    if (Nk(e, k) > 0) v += (T)Nk(e, k) * oo2ze * es(m + 1, em1(e, k));
                                    ep[m][e][k] = v;
                                }
                        if constexpr (LC == 1) {
#pragma unroll
                            for (int e = E0; e < E1; e++)
#pragma unroll
                                for (int k = 0; k < 3; k++) acc[e][1 + k] += ep[0][e][k];
                        }
                        if constexpr (FM == 2) {
                            const T oo2e = (T)0.5 * oe, re = rho * oe;
#pragma unroll
                            for (int e = E0; e < E1; e++)
#pragma unroll
                                for (int c6 = 0; c6 < 6; c6++) {
                                    const int k = DI(c6 + 4), l = DJ(c6 + 4);
                                    T v = QC[k] * ep[0][e][l] + WQ[k] * ep[1][e][l];
                                    if (k == l) v += oo2e * (es(0, e) - re * es(1, e));
                                    if (Nk(e, k) > 0) v += (T)Nk(e, k) * oo2ze * ep[1][em1(e, k)][l];
                                    acc[e][4 + c6] += v;
                                }
                        }
                    }
                }
            }
        }
    }
    // ---- HRR on the ket: |c d) from |f]
    constexpr int NA = LA ? 3 : 1, NB = LB ? 3 : 1, NC = LC ? 3 : 1, ND = LD ? 3 : 1;
    T kt[10][NC * ND];
#pragma unroll
    for (int e = E0; e < E1; e++) {
        if constexpr (LD == 0) {
#pragma unroll
            for (int ic = 0; ic < NC; ic++) kt[e][ic] = acc[e][LC ? 1 + ic : 0];
        } else {  // LC = LD = 1
#pragma unroll
            for (int k = 0; k < 3; k++)
#pragma unroll
                for (int l = 0; l < 3; l++) kt[e][k * 3 + l] = acc[e][dcomp(k, l)] + CD[l] * acc[e][1 + k];
        }
    }
    // ---- HRR on the bra and store
#pragma unroll
    for (int x = 0; x < NC * ND; x++) {
        if constexpr (LB == 0) {
#pragma unroll
            for (int i = 0; i < NA; i++) out[i * NC * ND + x] = kt[LA ? 1 + i : 0][x];
        } else {
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++)
                    out[(i * 3 + j) * NC * ND + x] = kt[dcomp(i, j)][x] + AB[j] * kt[1 + i][x];
        }
    }
}

}  // namespace eri
