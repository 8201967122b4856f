// Exchange-correlation quadrature on the molecular grid: AO values and
// gradients, density and its gradient, the B3LYP kernel, and the V_xc matrix.
//
// Paper: V_xc(rho) in Eq. 1 (Section 3.1), B3LYP only (Section 3.2), AO values
// recomputed on the grid instead of stored (Section 5, "Recomputation").
//   rho_p = sum_mn phi_pm D_mn phi_pn,  grad rho_p = 2 sum_mn grad phi_pm D_mn phi_pn,
//   E_xc = sum_p w_p e(rho_p, sigma_p),
//   V_xc = V' + V'^T,  V'_mn = sum_p phi_pm X_pn,
//   X_pn = w_p (v_rho/2 phi_pn + 2 v_sigma grad rho_p . grad phi_pn).
//
// One thread block owns one molecule's share of grid blocks (grid (nchunk,
// nmol)); per sub-block of BP points it evaluates every AO into shared memory,
// forms rho (G threads per point, shuffle-reduced), runs the functional in
// three parts on three full warps (lane = point), builds X, and accumulates V'
// in a per-thread register tile (16 x 16 threads, TILE x TILE entries each).
// V' and E_xc leave the block once, at the end.  TILE and NV (the density
// step's registers per thread) are sized for the launch's largest basis: on
// the FP64 path every issued DFMA costs the same whether or not its result is
// used (the pipe, not the issue, bounds the kernel).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "xc.cuh"
#include "boys.cuh"

template <typename T, typename TA, int BP, int TILE, int NV>
__global__ void __launch_bounds__(256, 1) grid_xc_kernel(DevBatch b, int nchunk, int mode, int skip_tc, int nbf_lo,
                                                          int nbf_hi) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = blockIdx.y, chunk = blockIdx.x;
    const MolDesc md = b.mol[m];
    if (mode == 0 && !b.st[m].active) return;
    if (skip_tc && b.mol[m].tcq) return;  // done by the tensor-core kernel
    if (md.nbf <= nbf_lo || md.nbf > nbf_hi) return;  // another size class's launch
    const int n = md.nbf, nsh = md.nsh;
    const int XS = n | 1;  // odd row stride of X (bank-conflict free both ways)
    T *Ds = (T *)smem_raw;                 // [n][n]
    T *phi = Ds + n * n;                   // [4][n][BP]
    T *Xs = phi + 4 * n * BP;              // [BP][XS]
    T *pt = Xs + BP * XS;                  // [4][BP] x y z w
    T *cf = pt + 4 * BP;                   // [4][BP] coefficients
    T *rr = cf + 4 * BP;                   // [4][BP] rho, grad rho
    T *xv = rr + 4 * BP;                   // [3][2][BP] v_rho, v_sigma per functional part
    T *shd = xv + 6 * BP;                  // [nsh][8]: x y z e0 e1 e2 (c's below)
    T *shc = shd + nsh * 8;                // [nsh][4]: c0 c1 c2 -
    T *dlt = shc + nsh * 4;                // [2][nsh][3]: R_owner - C_shell for the sub-block's owners
    int *shi = (int *)(dlt + 6 * nsh);     // [nsh][2]: l, ao0
    const double *D = b.mat + md.mat0 + (long long)M_D * n * n;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) Ds[i] = (T)D[i];
    for (int s = threadIdx.x; s < nsh; s += blockDim.x) {
        int g = md.sh0 + s;
        for (int k = 0; k < 3; k++) {
            shd[s * 8 + k] = (T)b.sh_xyz[g * 3 + k];
            shd[s * 8 + 3 + k] = (T)b.sh_ex[g * 3 + k];
            shc[s * 4 + k] = (T)b.sh_co[g * 3 + k];
        }
        shi[s * 2] = b.sh_l[g];
        shi[s * 2 + 1] = b.sh_ao0[g];
    }
    const int t = threadIdx.x;
    const int ti = t >> 4, tj = t & 15;
    TA acc[TILE][TILE];
#pragma unroll
    for (int a = 0; a < TILE; a++)
#pragma unroll
        for (int c = 0; c < TILE; c++) acc[a][c] = (TA)0;
    double exc = 0.0;
    constexpr int G = 256 / BP;  // threads per point in the density step
    const T *gx = (const T *)b.gx + md.pts0, *gy = (const T *)b.gy + md.pts0;
    const T *gz = (const T *)b.gz + md.pts0, *gw = (const T *)b.gw + md.pts0;
    const int nsub = md.nblk * (RKS_PTS_BLOCK / BP);
    const int npa = b.n_rad * b.n_theta * b.n_phi;
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
        // centre offsets for the (at most two) atoms owning this sub-block's points
        for (int i = t; i < 2 * nsh; i += blockDim.x) {
            const int h = i / nsh, s = i % nsh;
            const int A = min(own0 + h, md.natom - 1);
            const double *ra = b.axyz + (md.atom0 + A) * 3, *rc = b.sh_xyz + (md.sh0 + s) * 3;
            dlt[(h * nsh + s) * 3 + 0] = (T)(ra[0] - rc[0]);
            dlt[(h * nsh + s) * 3 + 1] = (T)(ra[1] - rc[1]);
            dlt[(h * nsh + s) * 3 + 2] = (T)(ra[2] - rc[2]);
        }
        __syncthreads();
        // ---- AO values and gradients: phi[0..3][mu][p]
        for (int idx = t; idx < nsh * BP; idx += blockDim.x) {
            const int s = idx / BP, p = idx % BP;
            const int h = min((int)((p0 + p) / npa), md.natom - 1) - own0;
            const T *dl = dlt + (h * nsh + s) * 3;
            const T dx = dl[0] + pt[p], dy = dl[1] + pt[BP + p], dz = dl[2] + pt[2 * BP + p];
            const T r2 = dx * dx + dy * dy + dz * dz;
            T g = 0, gp = 0;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const T x = shd[s * 8 + 3 + k] * r2;
                if (x < (T)40) {  // e^-40 ~ 4e-18: below anything the sums can see
                    const T e = shc[s * 4 + k] * xc::exp_(-x);
                    g += e;
                    gp -= (T)2 * shd[s * 8 + 3 + k] * e;
                }
            }
            const int l = shi[s * 2], mu = shi[s * 2 + 1];
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
        __syncthreads();
        // ---- density: G threads per point; thread gg owns a contiguous run of
        // NV columns nu of T = Phi D, summed in NV independent registers (the
        // FP64 pipe needs the independent chains to stay busy)
        {
            const int p = t / G, gg = t % G;
            const int nper = (n + G - 1) / G, nu0 = gg * nper;
            T tv[NV];
#pragma unroll
            for (int v = 0; v < NV; v++) tv[v] = (T)0;
            for (int mu = 0; mu < n; mu++) {
                const T f = phi[mu * BP + p];
                const T *drow = Ds + mu * n + nu0;
#pragma unroll
                for (int v = 0; v < NV; v++)
                    if (v < nper && nu0 + v < n) tv[v] += f * drow[v];
            }
            T rho = 0, rx = 0, ry = 0, rz = 0;
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const int nu = nu0 + v;
                if (v < nper && nu < n) {
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
        }
        __syncthreads();
        // ---- the functional: part (exchange, VWN5, LYP) = warp, point = lane
        if (t < 96) {
            const int part = t >> 5;
            for (int p = t & 31; p < BP; p += 32) {
                const T w = pt[3 * BP + p];
                T e = 0, vr = 0, vs = 0;
                if (w != (T)0) {
                    const T gx = rr[BP + p], gy = rr[2 * BP + p], gz = rr[3 * BP + p];
                    xc::b3lyp_part<T>(part, rr[p], gx * gx + gy * gy + gz * gz, e, vr, vs);
                }
                exc += (double)w * (double)e;
                xv[(part * 2) * BP + p] = vr;
                xv[(part * 2 + 1) * BP + p] = vs;
            }
        }
        __syncthreads();
        for (int p = t; p < BP; p += blockDim.x) {
            const T w = pt[3 * BP + p];
            const T vr = xv[p] + xv[2 * BP + p] + xv[4 * BP + p], vs = xv[BP + p] + xv[5 * BP + p];
            cf[p] = (T)0.5 * w * vr;
            cf[BP + p] = (T)2 * w * vs * rr[BP + p];
            cf[2 * BP + p] = (T)2 * w * vs * rr[2 * BP + p];
            cf[3 * BP + p] = (T)2 * w * vs * rr[3 * BP + p];
        }
        __syncthreads();
        // ---- X[p][nu]
        for (int idx = t; idx < n * BP; idx += blockDim.x) {
            const int nu = idx / BP, p = idx % BP;
            Xs[p * XS + nu] = cf[p] * phi[nu * BP + p] + cf[BP + p] * phi[(n + nu) * BP + p] +
                              cf[2 * BP + p] * phi[(2 * n + nu) * BP + p] + cf[3 * BP + p] * phi[(3 * n + nu) * BP + p];
        }
        __syncthreads();
        // ---- V'[mu][nu] += sum_p phi[mu][p] X[p][nu]; the sub-block sum is
        // formed in T and folded into the TA accumulator once per sub-block
        T part[TILE][TILE];
#pragma unroll
        for (int a = 0; a < TILE; a++)
#pragma unroll
            for (int c = 0; c < TILE; c++) part[a][c] = (T)0;
        for (int p = 0; p < BP; p++) {
            T fa[TILE], xb[TILE];
#pragma unroll
            for (int a = 0; a < TILE; a++) {
                const int mu = ti + 16 * a;
                fa[a] = mu < n ? phi[mu * BP + p] : (T)0;
            }
#pragma unroll
            for (int c = 0; c < TILE; c++) {
                const int nu = tj + 16 * c;
                xb[c] = nu < n ? Xs[p * XS + nu] : (T)0;
            }
#pragma unroll
            for (int a = 0; a < TILE; a++)
#pragma unroll
                for (int c = 0; c < TILE; c++) part[a][c] += fa[a] * xb[c];
        }
#pragma unroll
        for (int a = 0; a < TILE; a++)
#pragma unroll
            for (int c = 0; c < TILE; c++) acc[a][c] += (TA)part[a][c];
        __syncthreads();
    }
    // ---- flush V' and E_xc
    // FP64 accumulators for the FP64 path, fixed point for every pass of the mixed path
    using TG = std::conditional_t<sizeof(T) == 8, double, Fx>;
    TG *gV;
    if constexpr (sizeof(T) == 8) gV = b.accd + md.acc0 + 2 * n * n;
    else gV = b.accx + md.acc0 + 2 * n * n;
#pragma unroll
    for (int a = 0; a < TILE; a++)
#pragma unroll
        for (int c = 0; c < TILE; c++) {
            const int mu = ti + 16 * a, nu = tj + 16 * c;
            if (mu < n && nu < n && acc[a][c] != (TA)0) acc_add(&gV[mu * n + nu], acc[a][c]);
        }
    for (int o = 16; o > 0; o >>= 1) exc += __shfl_xor_sync(0xffffffffu, exc, o);
    if ((t & 31) == 0 && exc != 0.0) exc_add(&b.st[m].exc_fx, exc);
}

template <typename T, typename TA, int BP, int TILE, int NV>
static void launch_gx1(const DevBatch &b, int nchunk, int mode, int skip_tc, int nbf_lo, int nbf_hi, int max_nsh,
                       cudaStream_t s) {
    const int n = nbf_hi, XS = n | 1;
    size_t sm = sizeof(T) * ((size_t)n * n + 4ull * n * BP + (size_t)BP * XS + 18ull * BP + 18ull * max_nsh) +
                sizeof(int) * 2ull * max_nsh + 64;
    cudaFuncSetAttribute(grid_xc_kernel<T, TA, BP, TILE, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    grid_xc_kernel<T, TA, BP, TILE, NV><<<dim3(nchunk, b.nmol), 256, sm, s>>>(b, nchunk, mode, skip_tc, nbf_lo, nbf_hi);
}

// One launch per basis-size class (nbf <= 64, <= 80, <= 96) up to the batch's
// largest: the V' tile and the density registers are sized for the class
// (16 TILE >= nbf; NV >= nbf / G with G = 256 / BP threads per point), and
// each launch skips the molecules of the other classes
template <typename T, typename TA, int BP>
static void launch_gx(const DevBatch &b, int nchunk, int mode, int skip_tc, int max_nbf, int max_nsh, cudaStream_t s) {
    constexpr int G = 256 / BP;
    static_assert(RKS_NBF_SMALL <= 96, "tile classes cover nbf <= 96 (larger molecules: large.cu)");
    launch_gx1<T, TA, BP, 4, (64 + G - 1) / G>(b, nchunk, mode, skip_tc, 0, std::min(max_nbf, 64), max_nsh, s);
    if (max_nbf > 64)
        launch_gx1<T, TA, BP, 5, (80 + G - 1) / G>(b, nchunk, mode, skip_tc, 64, std::min(max_nbf, 80), max_nsh, s);
    if (max_nbf > 80) launch_gx1<T, TA, BP, 6, (96 + G - 1) / G>(b, nchunk, mode, skip_tc, 80, max_nbf, max_nsh, s);
}

void launch_grid_xc(const DevBatch &b, int nchunk, int acc_fp64, int mode, int skip_tc, int max_nbf, int max_nsh,
                    cudaStream_t s) {
    if (b.precision == 0) launch_gx<double, double, 32>(b, nchunk, mode, skip_tc, max_nbf, max_nsh, s);
    else if (acc_fp64) launch_gx<float, double, 64>(b, nchunk, mode, skip_tc, max_nbf, max_nsh, s);
    else launch_gx<float, float, 64>(b, nchunk, mode, skip_tc, max_nbf, max_nsh, s);
}

// --------------------------------------------------------- unit entry
template <typename T>
__global__ void eval_xc_kernel(int n, const double *rho, const double *sigma, double *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T e, vr, vs;
    xc::b3lyp<T>((T)rho[i], (T)sigma[i], e, vr, vs);
    out[3 * i] = e;
    out[3 * i + 1] = vr;
    out[3 * i + 2] = vs;
}

void launch_eval_xc(int n, const double *rho, const double *sigma, double *out, int fp32, cudaStream_t s) {
    if (fp32) eval_xc_kernel<float><<<(n + 127) / 128, 128, 0, s>>>(n, rho, sigma, out);
    else eval_xc_kernel<double><<<(n + 127) / 128, 128, 0, s>>>(n, rho, sigma, out);
}
