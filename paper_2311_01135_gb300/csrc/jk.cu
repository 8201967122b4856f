// Coulomb and exchange contractions from the packed two-electron store
// (paper Section 3.1, Eq. 1:  J_kl = sum_ij I_ijkl rho_ij,
// K_il = -1/2 sum_jk I_ijkl rho_jk; here K_std_il = sum_jk (ij|kl) rho_jk is
// accumulated and the -a0/2 factor is applied in the Fock assembly).
//
// The store holds one block per symmetry-distinct shell quartet (Section 3.2:
// 8-fold symmetry cuts storage and J/K flops by 8).  Each stored element v of a
// canonical quartet, scaled by 1/|stabiliser| (a factor 1/2 each for P = Q,
// R = S and pq = rs), stands for its 8 permutations:
//   J'_ij += 2 v D_kl,  J'_kl += 2 v D_ij,
//   K'_ik += v D_jl,  K'_jk += v D_il,  K'_il += v D_jk,  K'_jl += v D_ik,
// and J = J' + J'^T, K_std = K' + K'^T.
//
// The paper's IPU version replicated the density per thread and summed N^2
// partial vectors at the end (Section 5, "Current (Naive) Bottleneck").  Here
// one thread block owns one slice of one molecule's rows: D sits once in shared
// memory, a warp walks one row pq (lanes take consecutive rs), the row-local
// J'_PQ terms are reduced across the warp by shuffles, the K' terms that a run
// of kets with the same R shares are summed across that run's lanes, the
// remaining scattered terms go to shared-memory accumulators, and the block
// adds its J'/K' to the molecule's global accumulators once at the end.
#include "common.cuh"
#include "eri.cuh"
#include "kernels.h"

#define TAU_SCHWARZ 1e-12

// TA: arithmetic type of the contributions; TACC: accumulator (double, or
// the fixed-point Fx of the mixed iterations, whose sums do not depend on the
// order of the atomic adds).
// The K'_PR and K'_QR blocks are handed back in kpr_o / kqr_o for the
// caller's reduction over the run of kets that share R.
template <typename TS, typename TA, typename TACC, int LA, int LB, int LC, int LD>
__device__ __forceinline__ void jk_block(const TS *__restrict__ v, TA scale, int a0, int b0, int c0, int d0,
                                         const TA *Ds, TACC *Js, TACC *Ks, int n, TA *jpq, TA (&kpr_o)[3][3],
                                         TA (&kqr_o)[3][3]) {
    constexpr int na = LA ? 3 : 1, nb = LB ? 3 : 1, nc = LC ? 3 : 1, nd = LD ? 3 : 1;
    TA Drs[nc][nd], Dpq[na][nb], Dqs[nb][nd], Dps[na][nd], Dqr[nb][nc], Dpr[na][nc];
#pragma unroll
    for (int k = 0; k < nc; k++)
#pragma unroll
        for (int l = 0; l < nd; l++) Drs[k][l] = Ds[(c0 + k) * n + d0 + l];
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int j = 0; j < nb; j++) Dpq[i][j] = Ds[(a0 + i) * n + b0 + j];
#pragma unroll
    for (int j = 0; j < nb; j++)
#pragma unroll
        for (int l = 0; l < nd; l++) Dqs[j][l] = Ds[(b0 + j) * n + d0 + l];
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int l = 0; l < nd; l++) Dps[i][l] = Ds[(a0 + i) * n + d0 + l];
#pragma unroll
    for (int j = 0; j < nb; j++)
#pragma unroll
        for (int k = 0; k < nc; k++) Dqr[j][k] = Ds[(b0 + j) * n + c0 + k];
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int k = 0; k < nc; k++) Dpr[i][k] = Ds[(a0 + i) * n + c0 + k];

    TA jrs[nc][nd] = {}, kpr[na][nc] = {}, kqr[nb][nc] = {}, kps[na][nd] = {}, kqs[nb][nd] = {};
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int j = 0; j < nb; j++)
#pragma unroll
            for (int k = 0; k < nc; k++)
#pragma unroll
                for (int l = 0; l < nd; l++) {
                    const TA x = scale * (TA)v[((i * nb + j) * nc + k) * nd + l];
                    jpq[i * nb + j] += x * Drs[k][l];
                    jrs[k][l] += x * Dpq[i][j];
                    kpr[i][k] += x * Dqs[j][l];
                    kqr[j][k] += x * Dps[i][l];
                    kps[i][l] += x * Dqr[j][k];
                    kqs[j][l] += x * Dpr[i][k];
                }
#pragma unroll
    for (int k = 0; k < nc; k++)
#pragma unroll
        for (int l = 0; l < nd; l++) acc_add(&Js[(c0 + k) * n + d0 + l], (TA)2 * jrs[k][l]);
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int k = 0; k < nc; k++) kpr_o[i][k] = kpr[i][k];
#pragma unroll
    for (int j = 0; j < nb; j++)
#pragma unroll
        for (int k = 0; k < nc; k++) kqr_o[j][k] = kqr[j][k];
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int l = 0; l < nd; l++) acc_add(&Ks[(a0 + i) * n + d0 + l], kps[i][l]);
#pragma unroll
    for (int j = 0; j < nb; j++)
#pragma unroll
        for (int l = 0; l < nd; l++) acc_add(&Ks[(b0 + j) * n + d0 + l], kqs[j][l]);
}

// Elements of the store staged per warp and window (coalesced loads): up to
// 32 x 27 (a chunk of the largest staged blocks), fewer when the molecule's
// D/J/K leave less room; a window must hold one staged block.  16 warps for
// FP32 arithmetic, 8 for FP64 (whose blocks need twice the registers).
#define JK_WARPS_MAX 16
#define JK_SMEM_LIMIT 232448
#define JK_STAGE_BLOCK 27  // largest block that goes through the stage

// Per kept pair s of the molecule, in shared memory: its Schwarz factor and
// a packed descriptor: AO start of R (bits 0-6), of S (7-13), l_R (14),
// l_S (15), R == S (16).
__device__ __forceinline__ uint32_t jk_pinfo(int c0, int d0, int lR, int lS, int same) {
    return (uint32_t)c0 | ((uint32_t)d0 << 7) | ((uint32_t)lR << 14) | ((uint32_t)lS << 15) | ((uint32_t)same << 16);
}

// Shared-memory plan: D (n^2 TA), J' and K' (n^2 TACC each), the pair table
// (when it fits) and the per-warp stages; 16 warps, or 8 when D/J/K are large.
struct JkPlan {
    int warps, ch, pairs_in_smem;
    size_t bytes;
};
template <typename TS, typename TA, typename TACC> static JkPlan jk_plan(int n, int npair) {
    const size_t mats = (((size_t)n * n * sizeof(TA) + 15) & ~(size_t)15) + 2 * (size_t)n * n * sizeof(TACC);
    const size_t table = (((size_t)npair * sizeof(float) + 15) & ~(size_t)15) +
                         (((size_t)npair * sizeof(uint32_t) + 15) & ~(size_t)15);
    const int ch_max = 32 * JK_STAGE_BLOCK;  // a full chunk of the largest staged blocks
    JkPlan p;
    for (p.warps = sizeof(TA) == 8 ? JK_WARPS_MAX / 2 : JK_WARPS_MAX; p.warps >= 8; p.warps /= 2)
        for (p.pairs_in_smem = 1; p.pairs_in_smem >= 0; p.pairs_in_smem--) {
            const size_t fixed = mats + (p.pairs_in_smem ? table : 0);
            if (fixed >= JK_SMEM_LIMIT) continue;
            const long long ch = (long long)((JK_SMEM_LIMIT - fixed) / ((size_t)p.warps * sizeof(TS)));
            if (ch < 2 * JK_STAGE_BLOCK) continue;
            p.ch = (int)(ch < ch_max ? ch : ch_max);
            p.bytes = fixed + (size_t)p.warps * p.ch * sizeof(TS);
            return p;
        }
    p.warps = 0;  // does not fit: the caller reports it
    p.ch = 0;
    p.pairs_in_smem = 0;
    p.bytes = 0;
    return p;
}

// grid (nchunk, nmol); mode 0: only molecules still iterating, 1: all.
//
// A warp walks one row pq; lane L takes ket rs = s0 + L of a 32-ket chunk.
// The pair table (Schwarz factors, AO starts, angular momenta) is copied to
// shared memory once per block.  The row's kept blocks are contiguous in the
// store, so the warp copies a window of them into its shared-memory stage
// with coalesced loads (lane e reads element e, e + 32, ...), then every lane
// reads its own block from shared memory (block sizes 1, 3, 9, 27, 81 are
// odd: no bank conflicts).  A chunk whose blocks exceed one window is done in
// several windows, each holding whole blocks.
template <typename TS, typename TA, typename TACC>
__global__ void __launch_bounds__((sizeof(TA) == 8 ? JK_WARPS_MAX / 2 : JK_WARPS_MAX) * 32)
    jk_kernel(DevBatch b, int nchunk, int mode, int max_pair, int CH, int pairs_in_smem) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = blockIdx.y;
    const MolDesc md = b.mol[m];
    if (mode == 0 && !b.st[m].active) return;
    if (md.big) return;  // above RKS_NBF_SMALL: jk_large_kernel
    const int n = md.nbf, nn = n * n;
    const int npair = b.npair[m];
    TA *Ds = (TA *)smem_raw;
    size_t o = ((size_t)nn * sizeof(TA) + 15) & ~(size_t)15;
    TACC *Js = (TACC *)(smem_raw + o);
    TACC *Ks = Js + nn;
    o += 2 * (size_t)nn * sizeof(TACC);
    float *kqf = (float *)(smem_raw + o);  // Schwarz factors rounded to FP32 (screening, see below)
    const double *kq = b.kq + md.pair0;    // and exact, for the few kets near the threshold
    uint32_t *pinfo = nullptr;
    if (pairs_in_smem) {
        o += ((size_t)max_pair * sizeof(float) + 15) & ~(size_t)15;  // keeps the stage below 16-byte aligned
        pinfo = (uint32_t *)(smem_raw + o);
        o += ((size_t)max_pair * sizeof(uint32_t) + 15) & ~(size_t)15;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    TS *stg = (TS *)(smem_raw + o) + (size_t)warp * CH;
    const double *D = b.mat + md.mat0 + (long long)M_D * nn;
    for (int i = threadIdx.x; i < nn; i += blockDim.x) {
        Ds[i] = (TA)D[i];
        Js[i] = TACC{};
        Ks[i] = TACC{};
    }
    auto pair_of = [&](int i) -> uint32_t {
        const int2 rs = b.kpair[md.pair0 + i];
        const int R = md.sh0 + rs.x, S = md.sh0 + rs.y;
        return jk_pinfo(b.sh_ao0[R], b.sh_ao0[S], b.sh_l[R], b.sh_l[S], R == S);
    };
    if (pairs_in_smem) {
        for (int i = threadIdx.x; i < npair; i += blockDim.x) {
            kqf[i] = (float)kq[i];
            pinfo[i] = pair_of(i);
        }
    } else {
        kqf = nullptr;  // tables stay in global memory
    }
    __syncthreads();
    const TS *store = (const TS *)b.store + md.eri0;
    // rows are taken from a per-molecule queue shared by the molecule's
    // blocks, longest first (row r holds r + 1 kets; the p-shell rows come last)
    for (;;) {
        int q = 0;
        if (lane == 0) q = atomicAdd(&b.jk_next[m], 1);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= npair) break;
        const int r = npair - 1 - q;
        const uint32_t bi = pairs_in_smem ? pinfo[r] : pair_of(r);
        const double qpq = kq[r];
        const float qpqf = (float)qpq;
        const int a0 = bi & 127, b0 = (bi >> 7) & 127, lP = (bi >> 14) & 1, lQ = (bi >> 15) & 1;
        const TA bra_scale = (bi >> 16) & 1 ? (TA)0.5 : (TA)1;
        const int npq = (lP ? 3 : 1) * (lQ ? 3 : 1);
        long long base = b.row_off[md.pair0 + m + r];
        TA jpq[9] = {};
        for (int s0 = 0; s0 <= r; s0 += 32) {
            const int s = s0 + lane;
            bool keep = false;
            uint32_t ki = 0;
            int nel = 0;
            if (s <= r) {
                ki = pairs_in_smem ? pinfo[s] : pair_of(s);
                // the store kept the quartet iff Q_pq Q_rs >= tau in FP64; the
                // FP32 product is within 2e-7 of it, so it decides every ket
                // outside +-1e-5 of tau, and the FP64 test the rest
                const float pf = qpqf * (kqf ? kqf[s] : (float)kq[s]);
                const bool pass = pf > (float)(TAU_SCHWARZ * (1.0 + 1e-5))   ? true
                                  : pf < (float)(TAU_SCHWARZ * (1.0 - 1e-5)) ? false
                                                                             : qpq * kq[s] >= TAU_SCHWARZ;
                if (pass) {
                    keep = true;
                    nel = npq * ((ki >> 14) & 1 ? 3 : 1) * ((ki >> 15) & 1 ? 3 : 1);
                }
            }
            TA kpr_o[3][3] = {}, kqr_o[3][3] = {};
            int x = nel;  // inclusive prefix sum of block sizes over the chunk
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o2);
                if (lane >= o2) x += y;
            }
            const int tot = __shfl_sync(0xffffffffu, x, 31);
            const int start = x - nel;  // this lane's block, relative to the chunk
            auto run_block = [&](const TS *v) {
                TA scale = bra_scale;
                if ((ki >> 16) & 1) scale *= (TA)0.5;
                if (s == r) scale *= (TA)0.5;
                const int c0 = ki & 127, d0 = (ki >> 7) & 127;
                const int cls = (lP << 3) | (lQ << 2) | (((ki >> 14) & 1) << 1) | ((ki >> 15) & 1);
                switch (cls) {
                case 0x0: jk_block<TS, TA, TACC, 0, 0, 0, 0>(v, scale, a0, b0, c0, d0, Ds, Js, Ks, n, jpq, kpr_o, kqr_o); break;
                case 0x8: jk_block<TS, TA, TACC, 1, 0, 0, 0>(v, scale, a0, b0, c0, d0, Ds, Js, Ks, n, jpq, kpr_o, kqr_o); break;
                case 0xA: jk_block<TS, TA, TACC, 1, 0, 1, 0>(v, scale, a0, b0, c0, d0, Ds, Js, Ks, n, jpq, kpr_o, kqr_o); break;
                case 0xC: jk_block<TS, TA, TACC, 1, 1, 0, 0>(v, scale, a0, b0, c0, d0, Ds, Js, Ks, n, jpq, kpr_o, kqr_o); break;
                case 0xE: jk_block<TS, TA, TACC, 1, 1, 1, 0>(v, scale, a0, b0, c0, d0, Ds, Js, Ks, n, jpq, kpr_o, kqr_o); break;
                case 0xF: jk_block<TS, TA, TACC, 1, 1, 1, 1>(v, scale, a0, b0, c0, d0, Ds, Js, Ks, n, jpq, kpr_o, kqr_o); break;
                default: break;
                }
            };
            // (pp|pp) blocks (81 elements) are read by their lane straight from
            // the store: a window of them would leave most lanes idle.  They
            // are the chunk's last lanes (kets are ordered by class).
            const bool big = nel > JK_STAGE_BLOCK;
            if (__any_sync(0xffffffffu, big) && big) run_block(store + base + start);
            int first = 0;  // lanes below it are done
            while (first < 32) {
                const int w0 = __shfl_sync(0xffffffffu, start, first);
                const bool mine = lane >= first && !big && x <= w0 + CH;
                int wend = mine ? x : w0;
                for (int o2 = 16; o2 > 0; o2 >>= 1) wend = max(wend, __shfl_xor_sync(0xffffffffu, wend, o2));
                const TS *src = store + base + w0;
                for (int e = lane; e < wend - w0; e += 32) stg[e] = src[e];
                __syncwarp();
                if (mine && keep) run_block(stg + (start - w0));
                __syncwarp();
                const unsigned pend = __ballot_sync(0xffffffffu, lane >= first && !mine && !big);
                first = pend ? __ffs(pend) - 1 : 32;
            }
            {
                // K'_PR and K'_QR target shell R's columns, and kets are sorted
                // by (class, R, S): a run of lanes shares R and would hit the
                // same shared-memory words.  Sum each run across its lanes
                // (segmented scan in a fixed lane order, so the sum does not
                // depend on which warp takes the row) and let its last lane add.
                const int key = s <= r ? (int)(ki & 127) : 128 + lane;  // AO start of R
                const int prv = __shfl_up_sync(0xffffffffu, key, 1), nxt = __shfl_down_sync(0xffffffffu, key, 1);
                const bool tail = lane == 31 || nxt != key;
                const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prv != key);
                const int lo = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
                const int ncm = __any_sync(0xffffffffu, s <= r && ((ki >> 14) & 1)) ? 3 : 1;
                const int nc = (ki >> 14) & 1 ? 3 : 1, c0 = ki & 127;
                const int na = lP ? 3 : 1, nbq = lQ ? 3 : 1;
#pragma unroll
                for (int i = 0; i < 6; i++)
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        const bool onq = i >= 3;
                        const int ii = onq ? i - 3 : i;
                        if (ii >= (onq ? nbq : na) || k >= ncm) continue;  // warp-uniform
                        TA x = onq ? kqr_o[ii][k] : kpr_o[ii][k];
#pragma unroll
                        for (int d = 1; d < 32; d <<= 1) {
                            const TA y = __shfl_up_sync(0xffffffffu, x, d);
                            if (lane - d >= lo) x += y;
                        }
                        if (tail && s <= r && k < nc && x != (TA)0)
                            acc_add(&Ks[((onq ? b0 : a0) + ii) * n + c0 + k], x);
                    }
            }
            base += tot;
        }
        // the J'_PQ block is common to the whole row: reduce across the warp
#pragma unroll
        for (int k = 0; k < 9; k++) {
            TA t = jpq[k];
            for (int o2 = 16; o2 > 0; o2 >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o2);
            jpq[k] = t;
        }
        if (lane < npq) {
            const int i = lQ ? lane / 3 : lane, j = lQ ? lane % 3 : 0;
            TA val = jpq[0];
#pragma unroll
            for (int k = 1; k < 9; k++)
                if (k == lane) val = jpq[k];
            acc_add(&Js[(a0 + i) * n + b0 + j], (TA)2 * val);
        }
    }
    __syncthreads();
    TACC *gJ;
    if constexpr (std::is_same<TACC, double>::value) gJ = b.accd + md.acc0;
    else gJ = b.accx + md.acc0;
    TACC *gK = gJ + nn;
    for (int i = threadIdx.x; i < nn; i += blockDim.x) {
        const TACC j = Js[i], k = Ks[i];
        if (acc_nonzero(j)) acc_merge(&gJ[i], j);
        if (acc_nonzero(k)) acc_merge(&gK[i], k);
    }
}

template <typename TS, typename TA, typename TACC>
static int launch_jk_t(const DevBatch &b, int nchunk, int mode, int n, int max_pair, cudaStream_t s) {
    const JkPlan p = jk_plan<TS, TA, TACC>(n, max_pair);
    if (!p.warps) return -1;
    cudaFuncSetAttribute(jk_kernel<TS, TA, TACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.bytes);
    jk_kernel<TS, TA, TACC><<<dim3(nchunk, b.nmol), p.warps * 32, p.bytes, s>>>(b, nchunk, mode, max_pair, p.ch,
                                                                                p.pairs_in_smem);
    return 0;
}

int launch_jk(const DevBatch &b, int nchunk, int acc_fp64, int mode, int max_nbf, int max_pair, cudaStream_t s) {
    if (b.precision == 0) return launch_jk_t<double, double, double>(b, nchunk, mode, max_nbf, max_pair, s);
    // mixed path: fixed-point sums in every pass; the final step forms the
    // products in FP64 (FP64 D): with FP32 D and products its energy moved by
    // ~1e-5 Ha, which the iterations tolerate but the reported energy does not
    if (acc_fp64) return launch_jk_t<float, double, Fx>(b, nchunk, mode, max_nbf, max_pair, s);
    return launch_jk_t<float, float, Fx>(b, nchunk, mode, max_nbf, max_pair, s);
}

// ------------------------------------------- dense FP64 recompute lists
// The mixed path keeps an FP32 store.  For the final Fock build, every kept
// quartet whose Schwarz bound Q_pq Q_rs is at least fix_theta is recomputed in
// FP64 and the difference (I_64 - I_32) is contracted with D into the FP64
// J'/K' accumulators (on top of the FP32-store contraction accumulated in
// FP64).  Quartets below the threshold keep their FP32 values: their rounding
// error is bounded by ~1e-7 Q_pq Q_rs.
__device__ __forceinline__ int class_index(int cls) {
    // (lP lQ lR lS) bit code -> 0..5 in packing order
    return cls == 0x0 ? 0 : cls == 0x8 ? 1 : cls == 0xA ? 2 : cls == 0xC ? 3 : cls == 0xE ? 4 : 5;
}

// One block per molecule: every kept quartet with Q_pq Q_rs >= fix_theta is
// appended to its class list (row, column, store offset).
__global__ void __launch_bounds__(256) fix_list_kernel(DevBatch b) {
    const int m = blockIdx.x;
    const MolDesc md = b.mol[m];
    __shared__ int cnt[6];
    if (threadIdx.x < 6) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // molecules above RKS_NBF_SMALL recompute their listed quartets inside
    // jk_large_kernel: their lists stay empty
    const int npair = md.big ? 0 : b.npair[m];
    double qmax = 0.0;
    for (int i = lane; i < npair; i += 32) qmax = fmax(qmax, b.kq[md.pair0 + i]);
    for (int o = 16; o > 0; o >>= 1) qmax = fmax(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
    int4 *list = b.fixlist + (long long)m * 6 * RKS_FIX_CAP;
    for (int r = warp; r < npair; r += nwarp) {
        const double qpq = b.kq[md.pair0 + r];
        if (qpq * qmax < b.fix_theta) continue;
        const int2 pq = b.kpair[md.pair0 + r];
        const int lP = b.sh_l[md.sh0 + pq.x], lQ = b.sh_l[md.sh0 + pq.y];
        const int npq = (lP ? 3 : 1) * (lQ ? 3 : 1);
        long long base = b.row_off[md.pair0 + m + r];
        for (int s0 = 0; s0 <= r; s0 += 32) {
            const int s = s0 + lane;
            bool keep = false, fix = false;
            int nel = 0, ci = 0;
            if (s <= r) {
                const double prod = qpq * b.kq[md.pair0 + s];
                if (prod >= 1e-12) {
                    const int2 rs = b.kpair[md.pair0 + s];
                    const int lR = b.sh_l[md.sh0 + rs.x], lS = b.sh_l[md.sh0 + rs.y];
                    keep = true;
                    fix = prod >= b.fix_theta;
                    nel = npq * (lR ? 3 : 1) * (lS ? 3 : 1);
                    ci = class_index((lP << 3) | (lQ << 2) | (lR << 1) | lS);
                }
            }
            int x = nel;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            const int tot = __shfl_sync(0xffffffffu, x, 31);
            if (keep && fix) {
                const int pos = atomicAdd(&cnt[ci], 1);
                if (pos < RKS_FIX_CAP) {
                    const long long off = base + x - nel;
                    list[ci * RKS_FIX_CAP + pos] = make_int4(r, s, (int)(off & 0xffffffff), (int)(off >> 32));
                }
            }
            base += tot;
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        b.fixcount[m * 6 + threadIdx.x] = cnt[threadIdx.x];
        if (cnt[threadIdx.x] > RKS_FIX_CAP) atomicOr(&b.st[m].err_flag, 8);
    }
}

void launch_fix_list(const DevBatch &b, cudaStream_t s) { fix_list_kernel<<<b.nmol, 256, 0, s>>>(b); }

// Thread per listed quartet of class (LA LB LC LD): FP64 block from the FP64
// pair data minus the FP32 store block, contracted with the FP64 density and
// added to the FP64 J'/K' accumulators.
template <int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(128) jk_fix_kernel(DevBatch b, int ci, int mode, const int *mlist) {
    const int m = mlist ? mlist[blockIdx.y] : blockIdx.y;
    if (mode == 0 && !b.st[m].active) return;
    const int cntm = min(b.fixcount[m * 6 + ci], RKS_FIX_CAP);
    const MolDesc md = b.mol[m];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cntm; k += gridDim.x * blockDim.x) {
    const int4 e = b.fixlist[((long long)m * 6 + ci) * RKS_FIX_CAP + k];
    const int r = e.x, s = e.y;
    const long long off = (long long)(unsigned)e.z | ((long long)e.w << 32);
    const int2 pq = b.kpair[md.pair0 + r], rs = b.kpair[md.pair0 + s];
    const int P = md.sh0 + pq.x, Q = md.sh0 + pq.y, R = md.sh0 + rs.x, S = md.sh0 + rs.y;
    double AB[3], CD[3], AC[3];
#pragma unroll
    for (int x = 0; x < 3; x++) {
        AB[x] = b.sh_xyz[P * 3 + x] - b.sh_xyz[Q * 3 + x];
        CD[x] = b.sh_xyz[R * 3 + x] - b.sh_xyz[S * 3 + x];
        AC[x] = b.sh_xyz[P * 3 + x] - b.sh_xyz[R * 3 + x];
    }
    const eri::PrimPair<double> *pp = (const eri::PrimPair<double> *)b.pairprim64;
    constexpr int na = LA ? 3 : 1, nb = LB ? 3 : 1, nc = LC ? 3 : 1, nd = LD ? 3 : 1;
    constexpr int N = na * nb * nc * nd;
    double v[N];
    eri::quartet_pd<double, LA, LB, LC, LD>(pp + (long long)(md.pair0 + r) * 9, pp + (long long)(md.pair0 + s) * 9,
                                            AB, CD, AC, b.boys64, v);
    const float *v32 = (const float *)b.store + md.eri0 + off;
    double scale = 1.0;
    if (P == Q) scale *= 0.5;
    if (R == S) scale *= 0.5;
    if (r == s) scale *= 0.5;
#pragma unroll
    for (int x = 0; x < N; x++) v[x] = scale * (v[x] - (double)v32[x]);
    const int n = md.nbf;
    const double *D = b.mat + md.mat0 + (long long)M_D * n * n;
    Fx *gJ = b.accx + md.acc0, *gK = gJ + (long long)n * n;  // the mixed path's fixed-point accumulators
    const int a0 = b.sh_ao0[P], b0 = b.sh_ao0[Q], c0 = b.sh_ao0[R], d0 = b.sh_ao0[S];
    double jpq[na][nb] = {}, jrs[nc][nd] = {}, kpr[na][nc] = {}, kqr[nb][nc] = {}, kps[na][nd] = {}, kqs[nb][nd] = {};
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int j = 0; j < nb; j++)
#pragma unroll
            for (int kk = 0; kk < nc; kk++)
#pragma unroll
                for (int l = 0; l < nd; l++) {
                    const double x = v[((i * nb + j) * nc + kk) * nd + l];
                    jpq[i][j] += x * D[(c0 + kk) * n + d0 + l];
                    jrs[kk][l] += x * D[(a0 + i) * n + b0 + j];
                    kpr[i][kk] += x * D[(b0 + j) * n + d0 + l];
                    kqr[j][kk] += x * D[(a0 + i) * n + d0 + l];
                    kps[i][l] += x * D[(b0 + j) * n + c0 + kk];
                    kqs[j][l] += x * D[(a0 + i) * n + c0 + kk];
                }
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int j = 0; j < nb; j++) acc_add(&gJ[(a0 + i) * n + b0 + j], 2.0 * jpq[i][j]);
#pragma unroll
    for (int kk = 0; kk < nc; kk++)
#pragma unroll
        for (int l = 0; l < nd; l++) acc_add(&gJ[(c0 + kk) * n + d0 + l], 2.0 * jrs[kk][l]);
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int kk = 0; kk < nc; kk++) acc_add(&gK[(a0 + i) * n + c0 + kk], kpr[i][kk]);
#pragma unroll
    for (int j = 0; j < nb; j++)
#pragma unroll
        for (int kk = 0; kk < nc; kk++) acc_add(&gK[(b0 + j) * n + c0 + kk], kqr[j][kk]);
#pragma unroll
    for (int i = 0; i < na; i++)
#pragma unroll
        for (int l = 0; l < nd; l++) acc_add(&gK[(a0 + i) * n + d0 + l], kps[i][l]);
#pragma unroll
    for (int j = 0; j < nb; j++)
#pragma unroll
        for (int l = 0; l < nd; l++) acc_add(&gK[(b0 + j) * n + d0 + l], kqs[j][l]);
    }
}

void launch_jk_fix(const DevBatch &b, int mode, cudaStream_t s, const int *mlist, int nlist, int nchunk) {
    const dim3 g(mlist ? nchunk : 8, mlist ? nlist : b.nmol);  // grid-stride over each molecule's list
    if (g.y == 0) return;
    jk_fix_kernel<0, 0, 0, 0><<<g, 128, 0, s>>>(b, 0, mode, mlist);
    jk_fix_kernel<1, 0, 0, 0><<<g, 128, 0, s>>>(b, 1, mode, mlist);
    jk_fix_kernel<1, 0, 1, 0><<<g, 128, 0, s>>>(b, 2, mode, mlist);
    jk_fix_kernel<1, 1, 0, 0><<<g, 128, 0, s>>>(b, 3, mode, mlist);
    jk_fix_kernel<1, 1, 1, 0><<<g, 128, 0, s>>>(b, 4, mode, mlist);
    jk_fix_kernel<1, 1, 1, 1><<<g, 128, 0, s>>>(b, 5, mode, mlist);
}
