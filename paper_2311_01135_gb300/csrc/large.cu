// Larger molecules (a basis above RKS_NBF_SMALL functions, up to RKS_NBF_CAP:
// the 20-30-heavy-atom workload) and direct SCF.
//
// The shared-memory kernels hold D, J', K' (jk.cu) or D and the V' tile
// (gridxc.cu) of one molecule on chip, which caps them at 96 functions.  Here
// D is read from global memory (it stays in L2) and the sums go to the
// molecule's global accumulators:
//
//  * jk_large_kernel: J/K of Section 3.1, Eq. 1 with the 8-fold symmetry of
//    Section 3.2, a warp per kept bra pair, a lane per ket.  A quartet's block
//    comes from the packed store, or is recomputed on the spot (direct SCF:
//    the paper's "Recomputation", Section 5, used when the packed stores of a
//    batch do not fit in device memory), or, in the mixed final step, is
//    recomputed in FP64 when its Schwarz bound Q_pq Q_rs is at least
//    fix_theta (the small molecules' FP64 recompute list, without the list).
//  * grid_rho_large_kernel + grid_vxc_large_kernel: V_xc of Eq. 1 in two
//    passes.  The first forms rho and grad rho per point (T = Phi D with D
//    streamed through shared memory in row tiles), evaluates B3LYP and keeps
//    the four per-point coefficients of X in global memory; the second builds
//    V'_mn = sum_p phi_pm X_pn one row tile of V' per thread block, with
//    X_pn = c0_p phi_pn + c_p . grad phi_pn formed while the AO values are
//    evaluated.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "eri.cuh"
#include "kernels.h"
#include "xc.cuh"

#define LG_TAU 1e-12  // the Schwarz threshold of the packed store (same test, FP64)

// ---------------------------------------------------------------- J/K
enum { JKL_STORE = 0, JKL_STORE_FIX = 1, JKL_DIRECT = 2 };

// One kept quartet (P Q | R S) = rows r (bra pair) and s (ket pair): its
// block, scaled by 1/|stabiliser|, contracted with D into J' (the bra part
// into jpq, reduced over the row by the caller) and K' (global atomics).
template <typename TS, typename TA, typename TACC, int KIND, int LA, int LB, int LC, int LD>
__device__ __forceinline__ void jkl_quartet(const DevBatch &b, const MolDesc &md, int r, int s, int P, int Q, int R,
                                            int S, const TS *blk, bool fix, const void *pp, const void *tab,
                                            const double *__restrict__ D, TACC *gJ, TACC *gK, int n, TA *jpq) {
    constexpr int na = LA ? 3 : 1, nb = LB ? 3 : 1, nc = LC ? 3 : 1, nd = LD ? 3 : 1;
    constexpr int N = na * nb * nc * nd;
    TA v[N];
    TA scale = (TA)1;
    if (P == Q) scale *= (TA)0.5;
    if (R == S) scale *= (TA)0.5;
    if (r == s) scale *= (TA)0.5;
    // recompute (TS precision when direct; FP64 for the quartets the stored
    // path lists in its final step) or read the stored block
    auto recompute = [&](auto tag) {
        using TR = decltype(tag);
        TR AB[3], CD[3], AC[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            AB[k] = (TR)(b.sh_xyz[P * 3 + k] - b.sh_xyz[Q * 3 + k]);
            CD[k] = (TR)(b.sh_xyz[R * 3 + k] - b.sh_xyz[S * 3 + k]);
            AC[k] = (TR)(b.sh_xyz[P * 3 + k] - b.sh_xyz[R * 3 + k]);
        }
        const eri::PrimPair<TR> *ppr = (const eri::PrimPair<TR> *)pp;
        TR out[N];
        eri::quartet_pd<TR, LA, LB, LC, LD>(ppr + (long long)(md.pair0 + r) * 9, ppr + (long long)(md.pair0 + s) * 9,
                                            AB, CD, AC, (const TR *)tab, out);
#pragma unroll
        for (int x = 0; x < N; x++) v[x] = scale * (TA)out[x];
    };
    auto read_store = [&]() {
#pragma unroll
        for (int x = 0; x < N; x++) v[x] = scale * (TA)blk[x];
    };
    if constexpr (KIND == JKL_DIRECT) {
        recompute(TS{});
    } else if constexpr (KIND == JKL_STORE_FIX) {
        if (fix) recompute(double{});
        else read_store();
    } else {
        read_store();
    }
    const int a0 = b.sh_ao0[P], b0 = b.sh_ao0[Q], c0 = b.sh_ao0[R], d0 = b.sh_ao0[S];
    TA jrs[nc][nd] = {}, kpr[na][nc] = {}, kqr[nb][nc] = {}, kps[na][nd] = {}, kqs[nb][nd] = {};
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int j = 0; j < nb; j++)
#pragma unroll
            for (int k = 0; k < nc; k++)
#pragma unroll
                for (int l = 0; l < nd; l++) {
                    const TA x = v[((i * nb + j) * nc + k) * nd + l];
                    jpq[i * nb + j] += x * (TA)D[(c0 + k) * n + d0 + l];
                    jrs[k][l] += x * (TA)D[(a0 + i) * n + b0 + j];
                    kpr[i][k] += x * (TA)D[(b0 + j) * n + d0 + l];
                    kqr[j][k] += x * (TA)D[(a0 + i) * n + d0 + l];
                    kps[i][l] += x * (TA)D[(b0 + j) * n + c0 + k];
                    kqs[j][l] += x * (TA)D[(a0 + i) * n + c0 + k];
                }
#pragma unroll
    for (int k = 0; k < nc; k++)
#pragma unroll
        for (int l = 0; l < nd; l++) acc_add(&gJ[(c0 + k) * n + d0 + l], (TA)2 * jrs[k][l]);
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int k = 0; k < nc; k++) acc_add(&gK[(a0 + i) * n + c0 + k], kpr[i][k]);
#pragma unroll
    for (int j = 0; j < nb; j++)
#pragma unroll
        for (int k = 0; k < nc; k++) acc_add(&gK[(b0 + j) * n + c0 + k], kqr[j][k]);
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int l = 0; l < nd; l++) acc_add(&gK[(a0 + i) * n + d0 + l], kps[i][l]);
#pragma unroll
    for (int j = 0; j < nb; j++)
#pragma unroll
        for (int l = 0; l < nd; l++) acc_add(&gK[(b0 + j) * n + d0 + l], kqs[j][l]);
}

// grid (nchunk, nmol), 128 threads.  Rows (kept bra pairs) come from the
// molecule's queue, longest first; lanes take kets s = s0 + lane <= r, keep
// those with Q_pq Q_rs >= tau (the store's own test), and find their block's
// offset in the row by a warp prefix sum of the block sizes.  all_mol: every
// molecule (direct SCF); otherwise only those above RKS_NBF_SMALL.
template <typename TS, typename TA, typename TACC, int KIND>
__global__ void __launch_bounds__(128) jk_large_kernel(DevBatch b, int mode, int all_mol, const void *pp,
                                                        const void *tab) {
    const int m = blockIdx.y;
    const MolDesc md = b.mol[m];
    if (mode == 0 && !b.st[m].active) return;
    if (!all_mol && md.nbf <= RKS_NBF_SMALL) return;
    const int n = md.nbf, nn = n * n, lane = threadIdx.x & 31;
    const int npair = b.npair[m];
    const double *D = b.mat + md.mat0 + (long long)M_D * nn;
    TACC *gJ;
    if constexpr (std::is_same<TACC, double>::value) gJ = b.accd + md.acc0;
    else gJ = b.accx + md.acc0;
    TACC *gK = gJ + nn;
    const TS *store = KIND == JKL_DIRECT ? nullptr : (const TS *)b.store + md.eri0;
    const double *kq = b.kq + md.pair0;
    for (;;) {
        int q = 0;
        if (lane == 0) q = atomicAdd(&b.jk_next[m], 1);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= npair) break;
        const int r = npair - 1 - q;
        const int2 pq = b.kpair[md.pair0 + r];
        const int P = md.sh0 + pq.x, Q = md.sh0 + pq.y;
        const int lP = b.sh_l[P], lQ = b.sh_l[Q];
        const int npq = (lP ? 3 : 1) * (lQ ? 3 : 1);
        const double qpq = kq[r];
        long long base = KIND == JKL_DIRECT ? 0 : b.row_off[md.pair0 + m + r];
        TA jpq[9] = {};
        for (int s0 = 0; s0 <= r; s0 += 32) {
            const int s = s0 + lane;
            bool keep = false, fix = false;
            int R = 0, S = 0, lR = 0, lS = 0, nel = 0;
            if (s <= r) {
                const double prod = qpq * kq[s];
                if (prod >= LG_TAU) {
                    const int2 rs = b.kpair[md.pair0 + s];
                    R = md.sh0 + rs.x;
                    S = md.sh0 + rs.y;
                    lR = b.sh_l[R];
                    lS = b.sh_l[S];
                    keep = true;
                    fix = prod >= b.fix_theta;
                    nel = npq * (lR ? 3 : 1) * (lS ? 3 : 1);
                }
            }
            int x = nel;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            const int tot = __shfl_sync(0xffffffffu, x, 31);
            if (keep) {
                const TS *blk = store ? store + base + (x - nel) : nullptr;
                const int cls = (lP << 3) | (lQ << 2) | (lR << 1) | lS;
                switch (cls) {
#define JKL_CASE(C, A_, B_, C_, D_)                                                                              \
    case C: jkl_quartet<TS, TA, TACC, KIND, A_, B_, C_, D_>(b, md, r, s, P, Q, R, S, blk, fix, pp, tab, D, gJ, gK, n, \
                                                             jpq); break;
                JKL_CASE(0x0, 0, 0, 0, 0)
                JKL_CASE(0x8, 1, 0, 0, 0)
                JKL_CASE(0xA, 1, 0, 1, 0)
                JKL_CASE(0xC, 1, 1, 0, 0)
                JKL_CASE(0xE, 1, 1, 1, 0)
                JKL_CASE(0xF, 1, 1, 1, 1)
#undef JKL_CASE
                default: atomicOr(&b.st[m].err_flag, 2); break;  // class outside the packing order
                }
            }
            base += tot;
        }
        // J'_PQ is common to the whole row: reduce over the warp
#pragma unroll
        for (int k = 0; k < 9; k++) {
            TA t = jpq[k];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            jpq[k] = t;
        }
        if (lane < npq) {
            const int i = lQ ? lane / 3 : lane, j = lQ ? lane % 3 : 0;
            TA val = jpq[0];
#pragma unroll
            for (int k = 1; k < 9; k++)
                if (k == lane) val = jpq[k];
            acc_add(&gJ[(b.sh_ao0[P] + i) * n + b.sh_ao0[Q] + j], (TA)2 * val);
        }
    }
}

template <typename TS, typename TA, typename TACC, int KIND>
static void launch_jkl(const DevBatch &b, int nchunk, int mode, int all_mol, const void *pp, const void *tab,
                       cudaStream_t s) {
    jk_large_kernel<TS, TA, TACC, KIND><<<dim3(nchunk, b.nmol), 128, 0, s>>>(b, mode, all_mol, pp, tab);
}

int launch_jk_large(const DevBatch &b, int nchunk, int jk_fin, int mode, int direct, cudaStream_t s) {
    if (b.precision == 0) {
        if (direct) launch_jkl<double, double, double, JKL_DIRECT>(b, nchunk, mode, 1, b.pairprim, b.boys64, s);
        else launch_jkl<double, double, double, JKL_STORE>(b, nchunk, mode, 0, nullptr, nullptr, s);
        return 0;
    }
    if (!jk_fin) {
        if (direct) launch_jkl<float, float, Fx, JKL_DIRECT>(b, nchunk, mode, 1, b.pairprim, b.boys32, s);
        else launch_jkl<float, float, Fx, JKL_STORE>(b, nchunk, mode, 0, nullptr, nullptr, s);
        return 0;
    }
    // the mixed path's final-step precision: FP64 products; direct SCF
    // recomputes every quartet in FP64, the stored path the quartets with
    // Q_pq Q_rs >= fix_theta
    if (direct) {
        if (!b.pairprim64) return -1;
        launch_jkl<double, double, Fx, JKL_DIRECT>(b, nchunk, mode, 1, b.pairprim64, b.boys64, s);
    } else if (b.pairprim64 && b.fix_theta > 0.0) {
        launch_jkl<float, double, Fx, JKL_STORE_FIX>(b, nchunk, mode, 0, b.pairprim64, b.boys64, s);
    } else {
        launch_jkl<float, double, Fx, JKL_STORE>(b, nchunk, mode, 0, nullptr, nullptr, s);
    }
    return 0;
}

// ---------------------------------------------------------------- grid
// Shell data of one molecule in shared memory (T): [nsh][8] centre and
// exponents, [nsh][4] contraction coefficients, [2][nsh][3] R_owner - C_shell
// for the (at most two) atoms owning a sub-block's points, and [nsh][2] ints
// (l, first AO).
template <typename T> struct LgShells {
    T *shd, *shc, *dlt;
    int *shi;
};

template <typename T> __device__ __forceinline__ LgShells<T> lg_shells(T *base, int nsh) {
    LgShells<T> s;
    s.shd = base;
    s.shc = s.shd + nsh * 8;
    s.dlt = s.shc + nsh * 4;
    s.shi = (int *)(s.dlt + 6 * nsh);
    return s;
}
template <typename T> __host__ __device__ constexpr size_t lg_shell_bytes(int nsh) {
    return sizeof(T) * 18 * (size_t)nsh + sizeof(int) * 2 * (size_t)nsh;
}

template <typename T> __device__ void lg_load_shells(const DevBatch &b, const MolDesc &md, LgShells<T> sh) {
    for (int s = threadIdx.x; s < md.nsh; s += blockDim.x) {
        const int g = md.sh0 + s;
        for (int k = 0; k < 3; k++) {
            sh.shd[s * 8 + k] = (T)b.sh_xyz[g * 3 + k];
            sh.shd[s * 8 + 3 + k] = (T)b.sh_ex[g * 3 + k];
            sh.shc[s * 4 + k] = (T)b.sh_co[g * 3 + k];
        }
        sh.shi[s * 2] = b.sh_l[g];
        sh.shi[s * 2 + 1] = b.sh_ao0[g];
    }
}

// R_owner - C_shell for the two atoms that can own the points p0 .. p0 + BP - 1
// (points are stored as offsets from their own nucleus, so every point-to-shell
// vector is formed from FP64 coordinate differences plus the offset).
template <typename T> __device__ void lg_owner_offsets(const DevBatch &b, const MolDesc &md, LgShells<T> sh, int own0) {
    const int nsh = md.nsh;
    for (int i = threadIdx.x; i < 2 * nsh; i += blockDim.x) {
        const int h = i / nsh, s = i % nsh;
        const int A = min(own0 + h, md.natom - 1);
        const double *ra = b.axyz + (md.atom0 + A) * 3, *rc = b.sh_xyz + (md.sh0 + s) * 3;
        for (int k = 0; k < 3; k++) sh.dlt[(h * nsh + s) * 3 + k] = (T)(ra[k] - rc[k]);
    }
}

// Radial part of shell s at offset (dx, dy, dz) from its centre:
// g = sum_k c_k exp(-a_k r^2), gp = sum_k (-2 a_k) c_k exp(-a_k r^2).
template <typename T>
__device__ __forceinline__ void lg_radial(const LgShells<T> &sh, int s, T dx, T dy, T dz, T &g, T &gp) {
    const T r2 = dx * dx + dy * dy + dz * dz;
    g = 0;
    gp = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const T x = sh.shd[s * 8 + 3 + k] * r2;
        if (x < (T)40) {  // e^-40 ~ 4e-18: below anything the sums can see
            const T e = sh.shc[s * 4 + k] * xc::exp_(-x);
            g += e;
            gp -= (T)2 * sh.shd[s * 8 + 3 + k] * e;
        }
    }
}

// D in FP32 for the mixed path's grid pass, once per pass (b.gdt at acc0):
// the density pass then streams FP32 tiles, with no FP64-to-FP32 conversion
// (a slow FP64-pipe instruction on this GPU) in its inner loop.
__global__ void d_to_f32_kernel(DevBatch b, int mode) {
    const int m = blockIdx.y;
    const MolDesc md = b.mol[m];
    if (mode == 0 && !b.st[m].active) return;
    if (md.nbf <= RKS_NBF_SMALL) return;
    const long long nn = nbf2(md.nbf);
    const double *D = b.mat + md.mat0 + (long long)M_D * nn;
    float *dst = (float *)b.gdt + md.acc0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (float)D[i];
}

// Pass 1.  grid (nchunk, nmol), 256 threads; per sub-block of BP points:
// phi and grad phi of every AO into shared memory, T = Phi D with G = 256/BP
// threads per point (thread g takes the columns nu = g, g + G, ...; D comes
// through shared memory DT rows at a time, in T: the FP64 matrix itself, or
// its FP32 copy on the mixed path), rho and grad rho, the functional (three
// parts on three warps, as in the shared-memory kernel), and the coefficients
// (w v_rho / 2, 2 w v_sigma grad rho) of X for pass 2.
#define LG_DT 32
template <typename T, int BP, int NV>
__global__ void __launch_bounds__(256, 1) grid_rho_large_kernel(DevBatch b, int nchunk, int mode, T *cfg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = blockIdx.y, chunk = blockIdx.x;
    const MolDesc md = b.mol[m];
    if (mode == 0 && !b.st[m].active) return;
    if (md.nbf <= RKS_NBF_SMALL) return;
    const int n = md.nbf, nsh = md.nsh, t = threadIdx.x;
    constexpr int G = 256 / BP;
    T *phi = (T *)smem_raw;           // [4][n][BP]
    T *Dt = phi + 4 * n * BP;         // [LG_DT][n]
    T *pt = Dt + LG_DT * n;           // [4][BP]
    T *rr = pt + 4 * BP;              // [4][BP]
    T *xv = rr + 4 * BP;              // [6][BP]
    LgShells<T> sh = lg_shells<T>(xv + 6 * BP, nsh);
    lg_load_shells<T>(b, md, sh);
    const T *D;
    if constexpr (sizeof(T) == 8) D = (const T *)(b.mat + md.mat0 + (long long)M_D * n * n);
    else D = (const T *)b.gdt + md.acc0;
    const T *gx = (const T *)b.gx + md.pts0, *gy = (const T *)b.gy + md.pts0;
    const T *gz = (const T *)b.gz + md.pts0, *gw = (const T *)b.gw + md.pts0;
    T *cf = cfg + 4 * md.pts0;
    const int nsub = md.nblk * (RKS_PTS_BLOCK / BP);
    const int npa = b.n_rad * b.n_theta * b.n_phi;
    double exc = 0.0;
    __syncthreads();
    for (int sb = chunk; sb < nsub; sb += nchunk) {
        const long long p0 = (long long)sb * BP;
        const int own0 = min((int)(p0 / npa), md.natom - 1);
        for (int i = t; i < BP; i += blockDim.x) {
            pt[i] = gx[p0 + i];
            pt[BP + i] = gy[p0 + i];
            pt[2 * BP + i] = gz[p0 + i];
            pt[3 * BP + i] = gw[p0 + i];
        }
        lg_owner_offsets<T>(b, md, sh, own0);
        __syncthreads();
        for (int idx = t; idx < nsh * BP; idx += blockDim.x) {
            const int s = idx / BP, p = idx % BP;
            const int h = min((int)((p0 + p) / npa), md.natom - 1) - own0;
            const T *dl = sh.dlt + (h * nsh + s) * 3;
            const T dx = dl[0] + pt[p], dy = dl[1] + pt[BP + p], dz = dl[2] + pt[2 * BP + p];
            T g, gp;
            lg_radial<T>(sh, s, dx, dy, dz, g, gp);
            const int l = sh.shi[s * 2], mu = sh.shi[s * 2 + 1];
            if (l == 0) {
                phi[(0 * n + mu) * BP + p] = g;
                phi[(1 * n + mu) * BP + p] = gp * dx;
                phi[(2 * n + mu) * BP + p] = gp * dy;
                phi[(3 * n + mu) * BP + p] = gp * dz;
            } else {
                const T d[3] = {dx, dy, dz};
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    phi[(0 * n + mu + c) * BP + p] = d[c] * g;
#pragma unroll
                    for (int x = 0; x < 3; x++)
                        phi[((1 + x) * n + mu + c) * BP + p] = gp * d[c] * d[x] + (x == c ? g : (T)0);
                }
            }
        }
        // T[p][nu] = sum_mu phi[mu][p] D[mu][nu], nu = gg + G v
        const int p = t / G, gg = t % G;
        T tv[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) tv[v] = (T)0;
        for (int mt = 0; mt < n; mt += LG_DT) {
            const int rows = min(LG_DT, n - mt);
            __syncthreads();  // the previous tile is consumed (first pass: phi is written)
            for (int i = t; i < rows * n; i += blockDim.x) Dt[i] = D[(long long)mt * n + i];
            __syncthreads();
            for (int k = 0; k < rows; k++) {
                const T f = phi[(mt + k) * BP + p];
                const T *drow = Dt + k * n;
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    const int nu = gg + G * v;
                    if (nu < n) tv[v] += f * drow[nu];
                }
            }
        }
        T rho = 0, rx = 0, ry = 0, rz = 0;
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const int nu = gg + G * v;
            if (nu < n) {
                rho += tv[v] * phi[nu * BP + p];
                rx += tv[v] * phi[(n + nu) * BP + p];
                ry += tv[v] * phi[(2 * n + nu) * BP + p];
                rz += tv[v] * phi[(3 * n + nu) * BP + p];
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            rho += __shfl_xor_sync(0xffffffffu, rho, o);
            rx += __shfl_xor_sync(0xffffffffu, rx, o);
            ry += __shfl_xor_sync(0xffffffffu, ry, o);
            rz += __shfl_xor_sync(0xffffffffu, rz, o);
        }
        if (gg == 0) {
            rr[p] = rho;
            rr[BP + p] = (T)2 * rx;
            rr[2 * BP + p] = (T)2 * ry;
            rr[3 * BP + p] = (T)2 * rz;
        }
        __syncthreads();
        if (t < 96) {
            const int part = t >> 5;
            for (int q = t & 31; q < BP; q += 32) {
                const T w = pt[3 * BP + q];
                T e = 0, vr = 0, vs = 0;
                if (w != (T)0) {
                    const T ax = rr[BP + q], ay = rr[2 * BP + q], az = rr[3 * BP + q];
                    xc::b3lyp_part<T>(part, rr[q], ax * ax + ay * ay + az * az, e, vr, vs);
                }
                exc += (double)w * (double)e;
                xv[(part * 2) * BP + q] = vr;
                xv[(part * 2 + 1) * BP + q] = vs;
            }
        }
        __syncthreads();
        for (int q = t; q < BP; q += blockDim.x) {
            const T w = pt[3 * BP + q];
            const T vr = xv[q] + xv[2 * BP + q] + xv[4 * BP + q], vs = xv[BP + q] + xv[5 * BP + q];
            T *c = cf + (p0 + q) * 4;
            c[0] = (T)0.5 * w * vr;
            c[1] = (T)2 * w * vs * rr[BP + q];
            c[2] = (T)2 * w * vs * rr[2 * BP + q];
            c[3] = (T)2 * w * vs * rr[3 * BP + q];
        }
        // thread q reads only point q's pt, rr and xv here and rewrites only
        // point q's pt before the next barrier: no other thread's entries race
    }
    for (int o = 16; o > 0; o >>= 1) exc += __shfl_xor_sync(0xffffffffu, exc, o);
    if ((t & 31) == 0 && exc != 0.0) exc_add(&b.st[m].exc_fx, exc);
}

// Pass 2.  grid (nchunk, row tiles, nmol), 256 threads as 16 x 16; the block
// owns rows mu = r0 + ti + 16 a (a < TR) and every column nu = tj + 16 c
// (c < TC, 16 TC >= nbf) of V'.  Per sub-block: X[p][nu] for every AO and the
// row tile's phi[mu][p], then the register tile accumulates phi^T X (formed in
// T, folded into TA once per sub-block when TA is wider).
template <typename T, typename TA, int BP, int TR, int TC>
__global__ void __launch_bounds__(256, 1) grid_vxc_large_kernel(DevBatch b, int nchunk, int mode, const T *cfg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = blockIdx.z, chunk = blockIdx.x, r0 = blockIdx.y * 16 * TR;
    const MolDesc md = b.mol[m];
    if (mode == 0 && !b.st[m].active) return;
    if (md.nbf <= RKS_NBF_SMALL || r0 >= md.nbf) return;
    const int n = md.nbf, nsh = md.nsh, t = threadIdx.x, ti = t >> 4, tj = t & 15;
    constexpr int XS = (16 * TC) | 1;  // odd row stride (bank-conflict free both ways)
    T *Xs = (T *)smem_raw;             // [BP][XS]
    T *phr = Xs + BP * XS;             // [16 TR][BP]
    T *pt = phr + 16 * TR * BP;        // [4][BP]
    T *cf = pt + 4 * BP;               // [4][BP]
    LgShells<T> sh = lg_shells<T>(cf + 4 * BP, nsh);
    lg_load_shells<T>(b, md, sh);
    const T *gx = (const T *)b.gx + md.pts0, *gy = (const T *)b.gy + md.pts0;
    const T *gz = (const T *)b.gz + md.pts0, *gw = (const T *)b.gw + md.pts0;
    const T *cfm = cfg + 4 * md.pts0;
    const int nsub = md.nblk * (RKS_PTS_BLOCK / BP);
    const int npa = b.n_rad * b.n_theta * b.n_phi;
    TA acc[TR][TC];
#pragma unroll
    for (int a = 0; a < TR; a++)
#pragma unroll
        for (int c = 0; c < TC; c++) acc[a][c] = (TA)0;
    // columns beyond nbf and rows beyond the tile's stay zero
    for (int i = t; i < BP * XS; i += blockDim.x) Xs[i] = (T)0;
    for (int i = t; i < 16 * TR * BP; i += blockDim.x) phr[i] = (T)0;
    __syncthreads();
    for (int sb = chunk; sb < nsub; sb += nchunk) {
        const long long p0 = (long long)sb * BP;
        const int own0 = min((int)(p0 / npa), md.natom - 1);
        for (int i = t; i < BP; i += blockDim.x) {
            pt[i] = gx[p0 + i];
            pt[BP + i] = gy[p0 + i];
            pt[2 * BP + i] = gz[p0 + i];
            pt[3 * BP + i] = gw[p0 + i];
        }
        for (int i = t; i < 4 * BP; i += blockDim.x) cf[(i & 3) * BP + (i >> 2)] = cfm[p0 * 4 + i];
        lg_owner_offsets<T>(b, md, sh, own0);
        __syncthreads();
        for (int idx = t; idx < nsh * BP; idx += blockDim.x) {
            const int s = idx / BP, p = idx % BP;
            const int h = min((int)((p0 + p) / npa), md.natom - 1) - own0;
            const T *dl = sh.dlt + (h * nsh + s) * 3;
            const T dx = dl[0] + pt[p], dy = dl[1] + pt[BP + p], dz = dl[2] + pt[2 * BP + p];
            T g, gp;
            lg_radial<T>(sh, s, dx, dy, dz, g, gp);
            const int l = sh.shi[s * 2], mu = sh.shi[s * 2 + 1];
            const T c0 = cf[p], c1 = cf[BP + p], c2 = cf[2 * BP + p], c3 = cf[3 * BP + p];
            if (l == 0) {
                Xs[p * XS + mu] = c0 * g + gp * (c1 * dx + c2 * dy + c3 * dz);
                if (mu >= r0 && mu < r0 + 16 * TR) phr[(mu - r0) * BP + p] = g;
            } else {
                const T d[3] = {dx, dy, dz};
                const T cd = c1 * dx + c2 * dy + c3 * dz;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    // grad(d_c g) = gp d_c d + g e_c
                    const T cc = c == 0 ? c1 : (c == 1 ? c2 : c3);
                    Xs[p * XS + mu + c] = c0 * d[c] * g + gp * d[c] * cd + g * cc;
                    if (mu + c >= r0 && mu + c < r0 + 16 * TR) phr[(mu + c - r0) * BP + p] = d[c] * g;
                }
            }
        }
        __syncthreads();
        if constexpr (std::is_same<T, TA>::value) {
            for (int p = 0; p < BP; p++) {
                T fa[TR], xb[TC];
#pragma unroll
                for (int a = 0; a < TR; a++) fa[a] = phr[(ti + 16 * a) * BP + p];
#pragma unroll
                for (int c = 0; c < TC; c++) xb[c] = Xs[p * XS + tj + 16 * c];
#pragma unroll
                for (int a = 0; a < TR; a++)
#pragma unroll
                    for (int c = 0; c < TC; c++) acc[a][c] += fa[a] * xb[c];
            }
        } else {
            T part[TR][TC];
#pragma unroll
            for (int a = 0; a < TR; a++)
#pragma unroll
                for (int c = 0; c < TC; c++) part[a][c] = (T)0;
            for (int p = 0; p < BP; p++) {
                T fa[TR], xb[TC];
#pragma unroll
                for (int a = 0; a < TR; a++) fa[a] = phr[(ti + 16 * a) * BP + p];
#pragma unroll
                for (int c = 0; c < TC; c++) xb[c] = Xs[p * XS + tj + 16 * c];
#pragma unroll
                for (int a = 0; a < TR; a++)
#pragma unroll
                    for (int c = 0; c < TC; c++) part[a][c] += fa[a] * xb[c];
            }
#pragma unroll
            for (int a = 0; a < TR; a++)
#pragma unroll
                for (int c = 0; c < TC; c++) acc[a][c] += (TA)part[a][c];
        }
        __syncthreads();
    }
    using TG = std::conditional_t<sizeof(T) == 8, double, Fx>;
    TG *gV;
    if constexpr (sizeof(T) == 8) gV = b.accd + md.acc0 + 2 * n * n;
    else gV = b.accx + md.acc0 + 2 * n * n;
#pragma unroll
    for (int a = 0; a < TR; a++)
#pragma unroll
        for (int c = 0; c < TC; c++) {
            const int mu = r0 + ti + 16 * a, nu = tj + 16 * c;
            if (mu < n && nu < n && acc[a][c] != (TA)0) acc_add(&gV[mu * n + nu], acc[a][c]);
        }
}

static_assert(16 * 14 >= RKS_NBF_CAP, "the column tile covers the largest basis");

template <typename T, typename TA, int BPR, int BPV, int TR>
static int launch_lg(const DevBatch &b, int nchunk, int mode, int max_nbf, int max_nsh, void *cfg, cudaStream_t s) {
    constexpr int TC = 14, NV = (RKS_NBF_CAP + 256 / BPR - 1) / (256 / BPR);
    const int n = max_nbf;
    const size_t sm1 = sizeof(T) * (4ull * n * BPR + (size_t)LG_DT * n + 14ull * BPR) + lg_shell_bytes<T>(max_nsh) + 64;
    const size_t sm2 = sizeof(T) * ((size_t)BPV * ((16 * TC) | 1) + 16ull * TR * BPV + 8ull * BPV) +
                       lg_shell_bytes<T>(max_nsh) + 64;
    if (sm1 > 232448 || sm2 > 232448) return -1;
    if constexpr (sizeof(T) == 4) {
        if (!b.gdt) return -1;
        d_to_f32_kernel<<<dim3(32, b.nmol), 256, 0, s>>>(b, mode);
    }
    cudaFuncSetAttribute(grid_rho_large_kernel<T, BPR, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    grid_rho_large_kernel<T, BPR, NV><<<dim3(nchunk, b.nmol), 256, sm1, s>>>(b, nchunk, mode, (T *)cfg);
    cudaFuncSetAttribute(grid_vxc_large_kernel<T, TA, BPV, TR, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm2);
    const int ntile = (n + 16 * TR - 1) / (16 * TR);
    grid_vxc_large_kernel<T, TA, BPV, TR, TC><<<dim3(nchunk, ntile, b.nmol), 256, sm2, s>>>(b, nchunk, mode,
                                                                                             (const T *)cfg);
    return 0;
}

int launch_grid_xc_large(const DevBatch &b, int nchunk, int acc_fp64, int mode, int max_nbf, int max_nsh,
                         cudaStream_t s) {
    void *cfg = b.gcf;
    if (!cfg) return -1;
    if (b.precision == 0) return launch_lg<double, double, 16, 32, 4>(b, nchunk, mode, max_nbf, max_nsh, cfg, s);
    if (acc_fp64) return launch_lg<float, double, 32, 32, 4>(b, nchunk, mode, max_nbf, max_nsh, cfg, s);
    return launch_lg<float, float, 32, 32, 7>(b, nchunk, mode, max_nbf, max_nsh, cfg, s);
}
