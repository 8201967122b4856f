// Exchange-correlation quadrature with the two grid contractions on the
// tensor cores (tcgen05, kind::tf32, 3xTF32 split products, FP32 accumulators
// in tensor memory).  Same quantities as gridxc.cu (paper Section 3.1 V_xc,
// Section 3.2 B3LYP, AOs recomputed per block as in Section 5):
//   GEMM1  T = Phi D            (M = 128 points, N = K = np = 4 NQ)
//   rho_p = sum_n T_pn phi_pn,  grad rho_p = 2 sum_n T_pn grad phi_pn
//   GEMM2  V' += Phi^T X        (M = 128 AO rows, N = np, K = 128 points)
// Split products (Ootomo & Yokota 2022): a = a_hi + a_lo with a_hi the TF32
// rounding of a; a b ~= a_hi b_hi + a_hi b_lo + a_lo b_hi, accumulated in FP32.
// The b_lo tile follows the b_hi tile row for row, so a_hi [b_hi | b_lo] is
// one MMA of N = 2 np into two halves of the accumulator and a_lo b_hi a
// second one into the first half: two MMAs per K step (an MMA's issue, not
// its N, sets the pace at these sizes), and the halves are summed when the
// accumulator is read.
//
// Column order.  The kernel works in its own order of the AO basis (the
// molecule's column plan, built on the host, layout in common.cuh): thread
// quarter q owns columns q NQ .. q NQ + NQ - 1, made of units of five columns
// (a heavy atom's 1s, 2s, 2px, 2py, 2pz, or up to five hydrogens) and single
// hydrogen columns.  Which kind a unit is does not vary across a warp, and
// where each value sits is fixed at compile time, so the per-column work is
// straight-line code.  D is loaded in that order and V' is written back
// through the same map.
//
// Operand layouts (every tcgen05 TF32 operand is K-major):
//  * GEMM1 contracts over AOs: Phi as a [point][AO] tile and D as a [nu][mu]
//    tile of 8 x 16-byte core matrices (8 rows x 4 K values, 128 contiguous
//    bytes); the core of (row group g, K chunk c) sits at g * SG + c * 128,
//    SG = np / 4 * 128.  A thread writes its point's 4 AOs with one 16-byte store.
//  * GEMM2 contracts over points: Phi^T and X as [AO][point] tiles in the
//    128-byte swizzled layout: an atom is 8 AO rows x 32 points (1 KB), the
//    16-byte chunk c of row r sits at chunk position c ^ r, the four atoms of a
//    row group follow each other and row groups are 4 KB apart.  A warp (32
//    points, one AO) writes one 128-byte row with 32 scalar stores that hit
//    32 different banks, without the padding an unswizzled tile would need.
//    A K step of 8 points is 32 bytes inside an atom.
//
// One thread block (512 threads, one per SM) owns a contiguous 1/nchunk of a
// molecule's 128-point grid blocks and keeps the running sum of V' in tensor
// memory.
// Thread t serves point p = t % 128 and the column quarter q4 = t / 128; the
// radial values g, g' of its columns stay in its registers between phases.
// Per block:
//   A   radial values, unit by unit (an atom's 2s and 2p share one set of
//       exponentials): overlaps the previous block's GEMM2
//   B   the previous block's V' added to the running sum
//   C   Phi (hi, lo); one thread issues GEMM1
//   E   each thread reads its point's T row segment and forms its share of rho
//       and grad rho
//   F   B3LYP in three parts on three warp groups
//   G   Phi^T and X = w (v_rho/2 phi + 2 v_sigma grad rho . grad phi)
//       (hi, lo) into the GEMM2 tiles (over GEMM1's Phi tile, done with);
//       one thread issues GEMM2
// Which atoms matter in a block (AO screening) is decided once, when the
// grid is built (grid_mask_kernel), from the block's radius range.
// FINAL (the mixed final step) forms T on the CUDA cores instead of GEMM1.
// Waits on the MMA barriers are bounded: on expiry the block records an error
// flag, waits (bounded) once more, frees its tensor memory and returns.
#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "xc.cuh"

#define TC_BP 128
#define TC_NPMAX RKS_TC_NPMAX   // padded basis size this kernel handles
#define TC_TMEM_COLS 512
#define TC_TCOL 0               // TMEM columns of T (GEMM1: two halves of np columns)
#define TC_VCOL 160             // of V' (GEMM2, one block: two halves of np columns)
#define TC_SCOL 320             // and of the running sum of V' over the CTA's blocks
#define TC_SPIN_LIMIT 4000000  // polls before a wait gives up: >= ~40 ms, far above any MMA here
#define TC_THREADS 512
#define TC_SCREEN 1e-9f         // per-block AO screening threshold, iterations
#define TC_SCREEN_FINAL 1e-14f  // and final step

static_assert(RKS_TC_NATMAX < 64, "one 64-bit significance mask per block, bit 63 never set");
static_assert(TC_NPMAX / 4 == 20, "a thread owns at most 20 AO columns");

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (no swizzle, sm_100-family version bits).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::tf32 instruction descriptor: D F32, A/B TF32, both K-major, M and N.
__device__ __forceinline__ uint32_t idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
                 "l"(a), "l"(b), "r"(id), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// Bounded wait for the given phase; returns false on expiry.
__device__ __forceinline__ bool wait(uint64_t *bar, uint32_t phase) {
    uint32_t done = 0;
    for (int it = 0; it < TC_SPIN_LIMIT && !done; it++) {
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(phase)
                     : "memory");
    }
    return done != 0;
}

__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void split4(const float *v, float4 &hi, float4 &lo) {
    hi.x = tf32_hi(v[0]); hi.y = tf32_hi(v[1]); hi.z = tf32_hi(v[2]); hi.w = tf32_hi(v[3]);
    lo.x = v[0] - hi.x; lo.y = v[1] - hi.y; lo.z = v[2] - hi.z; lo.w = v[3] - hi.w;
}

// byte offset of element (row, k) in the core-matrix tile with row-group stride sg
__device__ __forceinline__ uint32_t coff(int row, int k, uint32_t sg) {
    return (uint32_t)(row >> 3) * sg + (uint32_t)(k >> 2) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

// byte offset of element (row, point) in a 128-byte-swizzled K-major tile of
// 128 points: atoms of 8 rows x 32 points, four per row group
__device__ __forceinline__ uint32_t soff(int row, int pt) {
    return (uint32_t)(row >> 3) * 4096u + (uint32_t)(pt >> 5) * 1024u + (uint32_t)(row & 7) * 128u +
           (uint32_t)((((pt >> 2) & 7) ^ (row & 7)) * 16) + (uint32_t)(pt & 3) * 4u;
}

// descriptor of a 128-byte-swizzled K-major tile (row groups 4 KB apart)
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    return sdesc(saddr, 16, 4096) | ((uint64_t)2 << 61);
}

}  // namespace tc

// Byte offsets inside the dynamic shared buffer.  GEMM1's Phi tiles and
// GEMM2's Phi^T / X tiles share one region (GEMM1 is done before the latter
// are written; the next block's Phi waits for GEMM2).  GEMM2's A operand
// reads M = 128 AO rows, past the np rows of a Phi^T tile into the tiles
// after it (rows >= np are discarded): the X tiles follow, so every read stays
// inside the buffer.  The rho partials alias the start of the region
// (written after GEMM1, read before the GEMM2 tiles are written).
struct TcSmem {
    uint32_t D_hi, D_lo, phi_hi, phi_lo, pt_hi, pt_lo, x_hi, x_lo, part, xcp, grd, atx, atf, perm;
    uint32_t total;
};

#define TC_NAT 64  // atom table entries: ids 0 .. 62, and 63 = empty slot (all zero)
#define TC_ATX 32  // floats per atom: float4s a1, c1, -2 a1 c1 (1s), a2, c2s, -2 a2 c2s, c2p, -2 a2 c2p (2s, 2p)

__host__ __device__ inline TcSmem tc_layout(int np) {
    TcSmem s;
    uint32_t o = 0;
    const uint32_t dsz = (uint32_t)np * np * 4, opsz = (uint32_t)TC_BP * np * 4;
    s.D_hi = o; o += dsz;
    s.D_lo = o; o += dsz;   // 8 np^2 bytes: the swizzled tiles below start 1 KB aligned
    s.phi_hi = o;
    s.phi_lo = o + opsz;
    s.pt_hi = o;            // swizzled tiles, np / 8 row groups of 4 KB = opsz bytes each
    s.pt_lo = o + opsz;
    s.x_hi = o + 2 * opsz;
    s.x_lo = o + 3 * opsz;
    o += 4 * opsz;
    s.part = s.pt_hi;                       // rho, grad rho partials per AO quarter (4 x 4 x 128 floats)
    s.xcp = o; o += 3 * 2 * TC_BP * 4;      // v_rho, v_sigma per XC part
    s.grd = o; o += 3 * TC_BP * 4;          // grad rho
    s.atx = o; o += TC_NAT * TC_ATX * 4;    // per atom: exponents and coefficients
    s.atf = o; o += TC_NAT * 8 * 4;         // per atom: R_owner0 - R_atom (3), pad, R_owner1 - R_atom (3), pad
    s.perm = o; o += (uint32_t)np * 4;      // AO index of each of the kernel's columns (-1 padding)
    // GEMM2's A operand reads 128 rows (16 row groups of 4 KB, plus the K
    // offset inside an atom) from the start of the Phi^T lo tile: for small
    // bases that runs past the tiles, so the buffer extends to cover it
    const uint32_t reach = s.pt_lo + 16u * 4096u + 1024u;
    s.total = o > reach ? o : reach;
    return s;
}

// W columns of this thread's TMEM lane row: the loads are issued together,
// one wait covers them, and each register passes through an empty asm after
// the wait so that no use of it is scheduled above the wait.
template <int W> __device__ __forceinline__ void tld_issue(uint32_t taddr, uint32_t *r) {
#pragma unroll
    for (int k = 0; k < W / 4; k++)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[4 * k]), "=r"(r[4 * k + 1]), "=r"(r[4 * k + 2]), "=r"(r[4 * k + 3])
                     : "r"(taddr + 4 * k));
}
template <int W> __device__ __forceinline__ void tld_done(uint32_t *r, float *v) {
#pragma unroll
    for (int i = 0; i < W; i++) {
        asm volatile("" : "+r"(r[i]));
        v[i] = __uint_as_float(r[i]);
    }
}
__device__ __forceinline__ void tld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
template <int W> __device__ __forceinline__ void tld(uint32_t taddr, float *v) {
    uint32_t r[W];
    tld_issue<W>(taddr, r);
    tld_wait();
    tld_done<W>(r, v);
}
template <int W> __device__ __forceinline__ void tst(uint32_t taddr, const float *v) {
#pragma unroll
    for (int k = 0; k < W / 4; k++)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr + 4 * k),
                     "r"(__float_as_uint(v[4 * k])), "r"(__float_as_uint(v[4 * k + 1])),
                     "r"(__float_as_uint(v[4 * k + 2])), "r"(__float_as_uint(v[4 * k + 3]))
                     : "memory");
}

// Lower bound on the distance from a shell centre to any point of a block:
// the points of owner h lie on atom-centred spheres with radii in [lo, hi],
// and the centre sits at distance d from that atom.
__device__ __forceinline__ float shell_rmin(float d, float lo, float hi) {
    return d > hi ? d - hi : (d < lo ? lo - d : 0.f);
}

// ------------------------------------------------------- block masks (setup)
// One thread block per 128-point grid block of a molecule the tensor-core
// kernel takes: bit A of mask[0] (iterations) / mask[1] (final step) is set
// when a shell of atom A may exceed the screening threshold somewhere in the
// block: |phi|, |grad phi| <= sum_k |c_k| e^(-a_k r^2) (1 + r + 2 a_k r^3),
// which decreases in r beyond r = 4 bohr for every STO-3G exponent, evaluated
// at the smallest distance from the shell centre to the block's points.
__global__ void __launch_bounds__(TC_BP) grid_mask_kernel(DevBatch b, const int *blk_mol,
                                                          unsigned long long *mask) {
    const long long gblk = blockIdx.x;
    const int m = blk_mol[gblk];
    const MolDesc md = b.mol[m];
    if (!md.tcq) return;
    __shared__ unsigned blk_r[4];  // radius range per owner (float bits; r >= 0 orders as unsigned)
    __shared__ unsigned long long abits[2];
    __shared__ int nsig[2][2];
    const int t = threadIdx.x, lane = t & 31;
    if (t < 4) blk_r[t] = (t & 1) ? 0u : 0x7f800000u;
    if (t < 2) abits[t] = 0ull;
    __syncthreads();
    const long long p0 = gblk * TC_BP - md.pts0;  // first point of the block, molecule-local
    const int npa = b.n_rad * b.n_theta * b.n_phi;
    const int own0 = min((int)(p0 / npa), md.natom - 1);
    const float *gx = (const float *)b.gx, *gy = (const float *)b.gy, *gz = (const float *)b.gz;
    const long long gi = gblk * TC_BP + t;
    const float x = gx[gi], y = gy[gi], z = gz[gi];
    const int h = min((int)((p0 + t) / npa), md.natom - 1) - own0;
    const unsigned rb = __float_as_uint(sqrtf(x * x + y * y + z * z));
    const unsigned lo0 = __reduce_min_sync(0xffffffffu, h == 0 ? rb : 0x7f800000u);
    const unsigned hi0 = __reduce_max_sync(0xffffffffu, h == 0 ? rb : 0u);
    const unsigned lo1 = __reduce_min_sync(0xffffffffu, h == 1 ? rb : 0x7f800000u);
    const unsigned hi1 = __reduce_max_sync(0xffffffffu, h == 1 ? rb : 0u);
    if (lane == 0) {
        atomicMin(&blk_r[0], lo0);
        atomicMax(&blk_r[1], hi0);
        atomicMin(&blk_r[2], lo1);
        atomicMax(&blk_r[3], hi1);
    }
    __syncthreads();
    if (t < md.nsh) {  // nsh <= nbf <= 80 for the molecules with a plan
        const int g = md.sh0 + t;
        float rmin = 3.4e38f;
#pragma unroll
        for (int hh = 0; hh < 2; hh++) {
            const float lo = __uint_as_float(blk_r[2 * hh]), hi = __uint_as_float(blk_r[2 * hh + 1]);
            if (lo > hi) continue;  // no point of this owner in the block
            const int A = min(own0 + hh, md.natom - 1);
            const double *ra = b.axyz + (md.atom0 + A) * 3, *rc = b.sh_xyz + g * 3;
            const float dx = (float)(ra[0] - rc[0]), dy = (float)(ra[1] - rc[1]), dz = (float)(ra[2] - rc[2]);
            rmin = fminf(rmin, shell_rmin(sqrtf(dx * dx + dy * dy + dz * dz), lo, hi));
        }
        bool on_it = true, on_fin = true;
        if (rmin >= 4.f) {
            float bound = 0.f;
            for (int k = 0; k < 3; k++) {
                const float a = (float)b.sh_ex[g * 3 + k];
                bound += fabsf((float)b.sh_co[g * 3 + k]) * __expf(-a * rmin * rmin) *
                         (1.f + rmin + 2.f * a * rmin * rmin * rmin);
            }
            on_it = bound > TC_SCREEN;
            on_fin = bound > TC_SCREEN_FINAL;
        }
        const unsigned long long bit = 1ull << b.sh_atom[g];
        if (on_it) atomicOr(&abits[0], bit);
        if (on_fin) atomicOr(&abits[1], bit);
    }
    __syncthreads();
    // significant AOs: 5 per heavy atom, 1 per hydrogen
    int ni = 0, nf = 0;
    if (t < md.natom) {
        const int nao = b.Z[md.atom0 + t] > 1 ? 5 : 1;
        ni = ((abits[0] >> t) & 1ull) ? nao : 0;
        nf = ((abits[1] >> t) & 1ull) ? nao : 0;
    }
    ni = __reduce_add_sync(0xffffffffu, ni);
    nf = __reduce_add_sync(0xffffffffu, nf);
    if (lane == 0 && t < 64) {
        nsig[0][t >> 5] = ni;
        nsig[1][t >> 5] = nf;
    }
    __syncthreads();
    if (t == 0) {
        mask[2 * gblk] = abits[0];
        mask[2 * gblk + 1] = abits[1];
        const double si = nsig[0][0] + nsig[0][1], sf = nsig[1][0] + nsig[1][1];
        atomicAdd(&b.st[m].grid_pairs[0], (double)TC_BP * si * si);
        atomicAdd(&b.st[m].grid_pairs[1], (double)TC_BP * sf * sf);
    }
}

__global__ void grid_pairs_reset_kernel(DevBatch b) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < b.nmol) b.st[m].grid_pairs[0] = b.st[m].grid_pairs[1] = 0.0;
}

void launch_grid_masks(const DevBatch &b, long long nblk_total, const int *blk_mol, cudaStream_t s) {
    grid_pairs_reset_kernel<<<(b.nmol + 127) / 128, 128, 0, s>>>(b);
    if (b.blk_mask) grid_mask_kernel<<<(unsigned)nblk_total, TC_BP, 0, s>>>(b, blk_mol, b.blk_mask);
}

// ------------------------------------------------------------ the kernel
// What a CTA keeps across its blocks (set up once, before the block loop).
struct TcCta {
    const MolDesc *md;
    TcSmem L;
    unsigned char *sm;
    const float *atx, *atf;
    const int *perm;
    float *part, *xcp, *grd;
    uint64_t *bar1, *bar2;
    int *s_fail;
    uint32_t su, sg, tT, tV, tS, lanes, id, id2;
    int m, chunk, nchunk, n, np, t, lane, warp, p, q4, c0;
};

// Radial values of a hydrogen slot (atom A) at the point:
// g = sum_k c_k e^(-a_k r^2), g' = sum_k -2 a_k c_k e^(-a_k r^2), zero when the
// atom is below the block's screen (the empty id's bit is never set).
__device__ __forceinline__ void tc_light(const float *atx, const float *atfp, uint32_t A, unsigned long long amask,
                                         float px, float py, float pz, float &g, float &gp) {
    const float4 dl = *(const float4 *)(atfp + A * 8);
    const float dx = dl.x + px, dy = dl.y + py, dz = dl.z + pz;
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float *e = atx + A * TC_ATX;
    const float4 a = *(const float4 *)e, c = *(const float4 *)(e + 4), mm = *(const float4 *)(e + 8);
    const float e0 = __expf(-a.x * r2), e1 = __expf(-a.y * r2), e2 = __expf(-a.z * r2);
    const bool on = (amask >> A) & 1ull;
    g = on ? c.x * e0 + c.y * e1 + c.z * e2 : 0.f;
    gp = on ? mm.x * e0 + mm.y * e1 + mm.z * e2 : 0.f;
}

// A heavy atom's unit: g[0..2] = g_1s, g_2s, g_2p and gp[0..2] their
// derivative factors (the 2s and 2p shells share one set of exponentials),
// and the offset d = r - R_A in g[3], g[4], gp[3].
__device__ __forceinline__ void tc_heavy(const float *atx, const float *atfp, uint32_t A, float px, float py,
                                         float pz, float *g, float *gp) {
    const float4 dl = *(const float4 *)(atfp + A * 8);
    const float dx = dl.x + px, dy = dl.y + py, dz = dl.z + pz;
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float *e = atx + A * TC_ATX;
    const float4 a1 = *(const float4 *)e, c1 = *(const float4 *)(e + 4), m1 = *(const float4 *)(e + 8);
    const float4 a2 = *(const float4 *)(e + 12), c2 = *(const float4 *)(e + 16), m2 = *(const float4 *)(e + 20);
    const float4 c3 = *(const float4 *)(e + 24), m3 = *(const float4 *)(e + 28);
    const float e0 = __expf(-a1.x * r2), e1 = __expf(-a1.y * r2), e2 = __expf(-a1.z * r2);
    const float f0 = __expf(-a2.x * r2), f1 = __expf(-a2.y * r2), f2 = __expf(-a2.z * r2);
    g[0] = c1.x * e0 + c1.y * e1 + c1.z * e2;
    gp[0] = m1.x * e0 + m1.y * e1 + m1.z * e2;
    g[1] = c2.x * f0 + c2.y * f1 + c2.z * f2;
    gp[1] = m2.x * f0 + m2.y * f1 + m2.z * f2;
    g[2] = c3.x * f0 + c3.y * f1 + c3.z * f2;
    gp[2] = m3.x * f0 + m3.y * f1 + m3.z * f2;
    g[3] = dx;
    g[4] = dy;
    gp[3] = dz;
    gp[4] = 0.f;
}

// G for one value of c0 & 7 (B = 0 or 4, known at compile time): Phi^T and X
// (hi, lo) of the thread's columns into the swizzled GEMM2 tiles.  With
// a = w v_rho / 2 and b = 2 w v_sigma grad rho: an s column has
// X = a g + g' (b . d); a p column c has X_c = d_c (a g + g' (b . d)) + b_c g.
template <int NQ, int B>
__device__ __forceinline__ void tc_write_gemm2(const TcCta &C, const uint32_t *uw, uint32_t rw, const float *g,
                                               const float *gp, const float *atfp, float px, float py, float pz,
                                               float a, float bx, float by, float bz) {
    constexpr int U = NQ / 5, R = NQ % 5;
    const uint32_t pc = (uint32_t)(C.p >> 2) & 7u;
    const uint32_t tbase = (uint32_t)(C.c0 >> 3) * 4096u + (uint32_t)(C.p >> 5) * 1024u + (uint32_t)(C.p & 3) * 4u;
    unsigned char *pth = C.sm + C.L.pt_hi + tbase, *ptl = C.sm + C.L.pt_lo + tbase;
    unsigned char *xh_ = C.sm + C.L.x_hi + tbase, *xl_ = C.sm + C.L.x_lo + tbase;
    auto put = [&](int j, float f, float x) {
        const int r = (B + j) & 7, grp = (B + j) >> 3;
        const uint32_t off = (uint32_t)grp * 4096u + (uint32_t)r * 128u + ((pc ^ (uint32_t)r) << 4);
        const float fh = tc::tf32_hi(f), xh = tc::tf32_hi(x);
        *(float *)(pth + off) = fh;
        *(float *)(ptl + off) = f - fh;
        *(float *)(xh_ + off) = xh;
        *(float *)(xl_ + off) = x - xh;
    };
    auto light = [&](int j, uint32_t A) {
        const float4 dl = *(const float4 *)(atfp + A * 8);
        const float bd = bx * (dl.x + px) + by * (dl.y + py) + bz * (dl.z + pz);
        put(j, g[j], a * g[j] + gp[j] * bd);
    };
#pragma unroll
    for (int k = 0; k < U; k++) {
        const int j = 5 * k;
        if (uw[k] >> 31) {
            const float dx = g[j + 3], dy = g[j + 4], dz = gp[j + 3];
            const float bd = bx * dx + by * dy + bz * dz;
            const float g2p = g[j + 2], sp = a * g2p + gp[j + 2] * bd;
            put(j, g[j], a * g[j] + gp[j] * bd);
            put(j + 1, g[j + 1], a * g[j + 1] + gp[j + 1] * bd);
            put(j + 2, dx * g2p, dx * sp + bx * g2p);
            put(j + 3, dy * g2p, dy * sp + by * g2p);
            put(j + 4, dz * g2p, dz * sp + bz * g2p);
        } else {
#pragma unroll
            for (int r = 0; r < 5; r++) light(j + r, (uw[k] >> (6 * r)) & 63u);
        }
    }
#pragma unroll
    for (int r = 0; r < R; r++) light(5 * U + r, (rw >> (6 * r)) & 63u);
}

// The block loop of one CTA for threads owning NQ columns each, then the
// flush of V' and E_xc.
template <typename TA, bool FINAL, int NQ>
__device__ __forceinline__ void tc_loop(const DevBatch &b, TcCta &C, const uint32_t *uw, uint32_t rw) {
    constexpr int U = NQ / 5, R = NQ % 5;
    const MolDesc &md = *C.md;
    const int t = C.t, p = C.p, lane = C.lane;
    const uint32_t phi_base = (uint32_t)(p >> 3) * C.sg + (uint32_t)(C.c0 >> 2) * 128u + (uint32_t)(p & 7) * 16u;
    uint32_t ph1 = 0, ph2 = 0;
    bool pending = false;  // a GEMM2 in flight whose V' is not yet in the running sum
    bool in1 = false;      // a GEMM1 in flight
    bool any_block = false, failed = false;
    double exc = 0.0;
    bool first = true;  // the running sum of V' in TMEM is not yet written

    const float *gxp = (const float *)b.gx + md.pts0, *gyp = (const float *)b.gy + md.pts0;
    const float *gzp = (const float *)b.gz + md.pts0, *gwp = (const float *)b.gw + md.pts0;
    const unsigned long long *bmask = b.blk_mask + 2 * (md.pts0 / TC_BP) + (FINAL ? 1 : 0);
    const int npa = b.n_rad * b.n_theta * b.n_phi;
    // the CTA's blocks are one contiguous run (the owner-atom table changes
    // about once per atom's worth of blocks, not every few blocks)
    const int blk0 = (int)((long long)md.nblk * C.chunk / C.nchunk);
    const int blk1 = (int)((long long)md.nblk * (C.chunk + 1) / C.nchunk);
    float nx = gxp[blk0 * TC_BP + p], ny = gyp[blk0 * TC_BP + p], nz = gzp[blk0 * TC_BP + p];
    float nw = gwp[blk0 * TC_BP + p];
    // the MMA operand descriptors at K step 0 (the tiles do not move); a K
    // step adds its byte offset / 16 to the start-address field, which cannot
    // carry out of its 14 bits (every shared-memory address is below 2^18)
    const uint64_t g1ah = tc::sdesc(C.su + C.L.phi_hi, 128, C.sg), g1al = tc::sdesc(C.su + C.L.phi_lo, 128, C.sg);
    const uint64_t g1bh = tc::sdesc(C.su + C.L.D_hi, 128, C.sg);  // D_lo follows as rows np .. 2 np - 1
    const uint64_t g2ah = tc::sdesc_sw128(C.su + C.L.pt_hi), g2al = tc::sdesc_sw128(C.su + C.L.pt_lo);
    const uint64_t g2bh = tc::sdesc_sw128(C.su + C.L.x_hi);  // X_lo follows as rows np .. 2 np - 1
    int atf_owner = -1;  // owner atom the atf table was built for
    float *atf_w = const_cast<float *>(C.atf);

    // the pending GEMM2's V' row segment added to the running sum (FP32
    // round-to-nearest across blocks; the tensor cores' accumulation only
    // spans one block): 8 columns per batch of loads, one wait per batch
    auto drain = [&]() -> bool {
        const bool ok = __syncthreads_and(C.warp != 0 || tc::wait(C.bar2, ph2));  // warp 0 polls, the rest block
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) return false;  // still pending: the exit path waits on the same phase
        ph2 ^= 1;
        auto batch = [&](auto wtag, int c) {
            constexpr int W = decltype(wtag)::value;
            uint32_t rv[W], rv2[W], rs[W];
            float v[W], v2[W], s[W];
            tld_issue<W>(C.tV + C.lanes + C.c0 + c, rv);
            tld_issue<W>(C.tV + C.lanes + C.np + C.c0 + c, rv2);
            if (!first) tld_issue<W>(C.tS + C.lanes + C.c0 + c, rs);
            tld_wait();
            tld_done<W>(rv, v);
            tld_done<W>(rv2, v2);
#pragma unroll
            for (int i = 0; i < W; i++) v[i] += v2[i];
            if (!first) {
                tld_done<W>(rs, s);
#pragma unroll
                for (int i = 0; i < W; i++) v[i] += s[i];
            }
            tst<W>(C.tS + C.lanes + C.c0 + c, v);
        };
#pragma unroll
        for (int c = 0; c + 8 <= NQ; c += 8) batch(std::integral_constant<int, 8>{}, c);
        if constexpr (NQ % 8 != 0) batch(std::integral_constant<int, 4>{}, NQ - 4);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        first = false;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        return true;
    };

    for (int blk = blk0; blk < blk1; blk++) {
        const int p0 = blk * TC_BP;
        const int own0 = min(p0 / npa, md.natom - 1);
        const float px = nx, py = ny, pz = nz, pw = nw;
        if (blk + 1 < blk1) {  // this thread's point of the next block
            const int i1 = p0 + TC_BP + p;
            nx = gxp[i1]; ny = gyp[i1]; nz = gzp[i1]; nw = gwp[i1];
        }
        const unsigned long long amask = bmask[2 * blk];
        if (amask == 0ull) continue;  // every AO below the screen: rho under the XC cutoff everywhere
        any_block = true;
        if (own0 != atf_owner) {  // R_owner - R_A for the block's (at most two) owners
            __syncthreads();
            for (int i = t; i < 2 * md.natom; i += TC_THREADS) {
                const int hh = i / md.natom, A = i % md.natom;
                const int O = min(own0 + hh, md.natom - 1);
                const double *ra = b.axyz + (md.atom0 + O) * 3, *rc = b.axyz + (md.atom0 + A) * 3;
                *(float4 *)(atf_w + A * 8 + hh * 4) =
                    make_float4((float)(ra[0] - rc[0]), (float)(ra[1] - rc[1]), (float)(ra[2] - rc[2]), 0.f);
            }
            atf_owner = own0;
            __syncthreads();
        }
        const int hp = min((p0 + p) / npa, md.natom - 1) - own0;
        const float *atfp = C.atf + hp * 4;

        // ---- A: radial values of the thread's columns, unit by unit
        float g[NQ], gp[NQ];
#pragma unroll
        for (int k = 0; k < U; k++) {
            const int j = 5 * k;
            if (uw[k] >> 31) {
                const uint32_t A = uw[k] & 63u;
                if ((amask >> A) & 1ull) {
                    tc_heavy(C.atx, atfp, A, px, py, pz, g + j, gp + j);
                } else {
#pragma unroll
                    for (int r = 0; r < 5; r++) g[j + r] = gp[j + r] = 0.f;
                }
            } else {
#pragma unroll
                for (int r = 0; r < 5; r++)
                    tc_light(C.atx, atfp, (uw[k] >> (6 * r)) & 63u, amask, px, py, pz, g[j + r], gp[j + r]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; r++)
            tc_light(C.atx, atfp, (rw >> (6 * r)) & 63u, amask, px, py, pz, g[5 * U + r], gp[5 * U + r]);
        // ---- B: the previous block's V'
        if (pending) {
            if (!drain()) {
                failed = true;
                break;
            }
            pending = false;
        }
        // ---- C: Phi (hi, lo) into the [point][AO] tile
#pragma unroll
        for (int kc = 0; kc < NQ / 4; kc++) {
            float v[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int j = kc * 4 + i, k = j / 5, r = j % 5;
                if (j < 5 * U && r >= 2) {  // a heavy unit's p column: d_c g_2p
                    const float dc = r == 2 ? g[5 * k + 3] : (r == 3 ? g[5 * k + 4] : gp[5 * k + 3]);
                    v[i] = (uw[k] >> 31) ? dc * g[5 * k + 2] : g[j];
                } else {
                    v[i] = g[j];
                }
            }
            float4 hi, lo;
            tc::split4(v, hi, lo);
            *(float4 *)(C.sm + C.L.phi_hi + phi_base + kc * 128) = hi;
            *(float4 *)(C.sm + C.L.phi_lo + phi_base + kc * 128) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        float Tv[NQ];  // this thread's T columns
        if constexpr (!FINAL) {
            if (t == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int s = 0; s < C.np / 8; s++) {
                    const uint64_t ka = (uint64_t)s * 16u;  // 2 cores of 128 B, in 16-byte units
                    tc::mma(C.tT, g1ah + ka, g1bh + ka, C.id2, s > 0);  // [Phi_hi D_hi | Phi_hi D_lo]
                    tc::mma(C.tT, g1al + ka, g1bh + ka, C.id, 1);       // + Phi_lo D_hi into the first half
                }
                tc::commit(C.bar1);
            }
            in1 = true;
            const bool ok1 = __syncthreads_and(C.warp != 0 || tc::wait(C.bar1, ph1));
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!ok1) {
                failed = true;
                break;
            }
            ph1 ^= 1;
            in1 = false;
            // T = the two halves of the accumulator, 8 columns per batch of loads
            auto tbatch = [&](auto wtag, int c) {
                constexpr int W = decltype(wtag)::value;
                uint32_t r1[W], r2[W];
                float v2[W];
                tld_issue<W>(C.tT + C.lanes + C.c0 + c, r1);
                tld_issue<W>(C.tT + C.lanes + C.np + C.c0 + c, r2);
                tld_wait();
                tld_done<W>(r1, Tv + c);
                tld_done<W>(r2, v2);
#pragma unroll
                for (int i = 0; i < W; i++) Tv[c + i] += v2[i];
            };
#pragma unroll
            for (int c = 0; c + 8 <= NQ; c += 8) tbatch(std::integral_constant<int, 8>{}, c);
            if constexpr (NQ % 8 != 0) tbatch(std::integral_constant<int, 4>{}, NQ - 4);
        } else {
            // T on the CUDA cores: this point's row of Phi (hi + lo is the FP32
            // value) against D's rows, the thread's column quarter
#pragma unroll
            for (int j = 0; j < NQ; j++) Tv[j] = 0.f;
            const float *Dp = (const float *)(C.sm + C.L.D_hi);
            const uint32_t rowb = (uint32_t)(p >> 3) * C.sg + (uint32_t)(p & 7) * 16u;
            for (int mc = 0; mc < C.np / 4; mc++) {
                const float4 h4 = *(const float4 *)(C.sm + C.L.phi_hi + rowb + mc * 128);
                const float4 l4 = *(const float4 *)(C.sm + C.L.phi_lo + rowb + mc * 128);
                const float ph[4] = {h4.x + l4.x, h4.y + l4.y, h4.z + l4.z, h4.w + l4.w};
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const float4 *drow = (const float4 *)(Dp + (mc * 4 + i) * C.np + C.c0);
#pragma unroll
                    for (int k = 0; k < NQ / 4; k++) {
                        const float4 d4 = drow[k];
                        Tv[4 * k] += ph[i] * d4.x;
                        Tv[4 * k + 1] += ph[i] * d4.y;
                        Tv[4 * k + 2] += ph[i] * d4.z;
                        Tv[4 * k + 3] += ph[i] * d4.w;
                    }
                }
            }
            __syncthreads();  // every thread's reads of the Phi tile precede the partials written over it
        }
        // ---- E: this thread's share of rho and grad rho / 2:
        // s column: rho += g T, grad += g' T d; heavy unit with u = T_p . d:
        // rho += g_2p u, grad += g_2p' u d + g_2p T_p
        {
            float rho = 0.f, rx = 0.f, ry = 0.f, rz = 0.f;
            auto light = [&](int j, uint32_t A) {
                const float4 dl = *(const float4 *)(atfp + A * 8);
                const float s = gp[j] * Tv[j];
                rho += g[j] * Tv[j];
                rx += s * (dl.x + px);
                ry += s * (dl.y + py);
                rz += s * (dl.z + pz);
            };
#pragma unroll
            for (int k = 0; k < U; k++) {
                const int j = 5 * k;
                if (uw[k] >> 31) {
                    const float dx = g[j + 3], dy = g[j + 4], dz = gp[j + 3];
                    const float t2 = Tv[j + 2], t3 = Tv[j + 3], t4 = Tv[j + 4];
                    const float u = dx * t2 + dy * t3 + dz * t4;
                    rho += g[j] * Tv[j] + g[j + 1] * Tv[j + 1] + g[j + 2] * u;
                    const float s = gp[j] * Tv[j] + gp[j + 1] * Tv[j + 1] + gp[j + 2] * u;
                    rx += s * dx + g[j + 2] * t2;
                    ry += s * dy + g[j + 2] * t3;
                    rz += s * dz + g[j + 2] * t4;
                } else {
#pragma unroll
                    for (int r = 0; r < 5; r++) light(j + r, (uw[k] >> (6 * r)) & 63u);
                }
            }
#pragma unroll
            for (int r = 0; r < R; r++) light(5 * U + r, (rw >> (6 * r)) & 63u);
            C.part[(C.q4 * 4 + 0) * TC_BP + p] = rho;
            C.part[(C.q4 * 4 + 1) * TC_BP + p] = rx;
            C.part[(C.q4 * 4 + 2) * TC_BP + p] = ry;
            C.part[(C.q4 * 4 + 3) * TC_BP + p] = rz;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        // ---- F: XC in three parts on three warp groups (exchange, VWN5, LYP)
        if (t < 3 * TC_BP) {
            const int gi = t >> 7;
            float r = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
            for (int gq = 0; gq < 4; gq++) {
                r += C.part[(gq * 4 + 0) * TC_BP + p];
                gx += C.part[(gq * 4 + 1) * TC_BP + p];
                gy += C.part[(gq * 4 + 2) * TC_BP + p];
                gz += C.part[(gq * 4 + 3) * TC_BP + p];
            }
            gx *= 2.f; gy *= 2.f; gz *= 2.f;
            float e = 0.f, vr = 0.f, vs = 0.f;
            if (pw != 0.f) xc::b3lyp_part<float>(gi, r, gx * gx + gy * gy + gz * gz, e, vr, vs);
            exc += (double)pw * (double)e;
            C.xcp[(gi * 2 + 0) * TC_BP + p] = vr;
            C.xcp[(gi * 2 + 1) * TC_BP + p] = vs;
            if (gi == 0) {
                C.grd[p] = gx;
                C.grd[TC_BP + p] = gy;
                C.grd[2 * TC_BP + p] = gz;
            }
        }
        __syncthreads();
        // ---- G: Phi^T and X = a phi + b . grad phi with a = w v_rho / 2, b = 2 w v_sigma grad rho
        {
            const float vr = C.xcp[p] + C.xcp[2 * TC_BP + p] + C.xcp[4 * TC_BP + p];
            const float vs2 = 2.f * pw * (C.xcp[TC_BP + p] + C.xcp[5 * TC_BP + p]);
            const float a = 0.5f * pw * vr;
            const float bx = vs2 * C.grd[p], by = vs2 * C.grd[TC_BP + p], bz = vs2 * C.grd[2 * TC_BP + p];
            if (C.c0 & 4) tc_write_gemm2<NQ, 4>(C, uw, rw, g, gp, atfp, px, py, pz, a, bx, by, bz);
            else tc_write_gemm2<NQ, 0>(C, uw, rw, g, gp, atfp, px, py, pz, a, bx, by, bz);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        // ---- H: GEMM2 over the block's 128 points (K steps of 8 points: 32 bytes in an atom)
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int k = 0; k < TC_BP / 8; k++) {
                const uint64_t ko = (uint64_t)((k >> 2) * 64 + (k & 3) * 2);  // (k/4) KB + (k%4) 32 B, 16-byte units
                tc::mma(C.tV, g2ah + ko, g2bh + ko, C.id2, k > 0);  // [Phi_hi^T X_hi | Phi_hi^T X_lo]
                tc::mma(C.tV, g2al + ko, g2bh + ko, C.id, 1);       // + Phi_lo^T X_hi into the first half
            }
            tc::commit(C.bar2);
        }
        pending = true;
    }
    if (!failed && pending) {
        failed = !drain();
        if (!failed) pending = false;
    }
    if (failed && t == 0) *C.s_fail = 1;
    __syncthreads();
    // ---- flush V' (row mu = this thread's lane row, columns of its quarter)
    // into the molecule's AO order, and E_xc
    if (!*C.s_fail && any_block && !first) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int mu = (C.warp & 3) * 32 + lane;
        const int Pm = mu < C.np ? C.perm[mu] : -1;
        Fx *gV = b.accx + md.acc0 + 2 * C.n * C.n;  // mixed path: fixed point in every pass
        float v[NQ];
        tld<NQ>(C.tS + C.lanes + C.c0, v);
#pragma unroll
        for (int j = 0; j < NQ; j++) {
            const int Pn = C.perm[C.c0 + j];
            if (Pm >= 0 && Pn >= 0 && v[j] != 0.f) acc_add(&gV[Pm * C.n + Pn], (TA)v[j]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) exc += __shfl_xor_sync(0xffffffffu, exc, o);
    if (lane == 0 && exc != 0.0) exc_add(&b.st[C.m].exc_fx, exc);
    if (*C.s_fail && t == 0) {
        atomicOr(&b.st[C.m].err_flag, 4);
        // give in-flight MMAs a bounded chance to drain before freeing tensor memory
        if (in1) tc::wait(C.bar1, ph1);
        if (pending) tc::wait(C.bar2, ph2);
    }
}

// FINAL (the mixed path's final step, TA = double): the density contraction
// T = Phi D runs on the CUDA cores in FP32 with round-to-nearest sums (the
// tensor cores' truncating accumulation would bias rho and E_xc), V_xc stays
// on the tensor cores (it only moves the final eigenvalues, at ~1e-7), and
// V_xc is accumulated in 64-bit fixed point like every mixed pass.
// One instantiation per NQ (columns per thread quarter), launched over the
// molecules of that class only (list), so that each gets its own register
// allocation and shared-memory size.
template <typename TA, bool FINAL, int NQ>
__global__ void __launch_bounds__(TC_THREADS, 1) grid_xc_tc_kernel(DevBatch b, int nchunk, int mode, const int *list) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar1, bar2;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;
    const int m = list[blockIdx.y], chunk = blockIdx.x;
    const MolDesc md = b.mol[m];
    if (mode == 0 && !b.st[m].active) return;
    if ((long long)md.nblk * (chunk + 1) / nchunk == (long long)md.nblk * chunk / nchunk) return;  // no blocks
    TcCta C;
    C.md = &md;
    C.m = m;
    C.chunk = chunk;
    C.nchunk = nchunk;
    C.n = md.nbf;
    C.np = 4 * NQ;
    C.L = tc_layout(C.np);
    C.t = threadIdx.x;
    C.lane = C.t & 31;
    C.warp = C.t >> 5;
    C.p = C.t & (TC_BP - 1);
    C.q4 = C.t >> 7;
    C.c0 = C.q4 * NQ;
    C.sm = smem;
    C.part = (float *)(smem + C.L.part);
    C.xcp = (float *)(smem + C.L.xcp);
    C.grd = (float *)(smem + C.L.grd);
    float *atx = (float *)(smem + C.L.atx), *atf = (float *)(smem + C.L.atf);
    int *perm = (int *)(smem + C.L.perm);
    C.atx = atx;
    C.atf = atf;
    C.perm = perm;
    C.sg = (uint32_t)(C.np / 4) * 128u;  // bytes per 8-row group of the unswizzled tiles
    C.bar1 = &bar1;
    C.bar2 = &bar2;
    C.s_fail = &s_fail;
    const int n = C.n, nsh = md.nsh, np = C.np, t = C.t;
    const int *plan = b.tc_plan + (long long)m * RKS_TC_PLAN;

    // ---- per-CTA constants: the column plan, the atom tables, and D in the
    // kernel's column order (hi, lo) as GEMM1's B, or plain FP32 D for the
    // CUDA-core contraction of the final step
    for (int i = t; i < TC_NAT * TC_ATX; i += blockDim.x) atx[i] = 0.f;
    for (int i = t; i < TC_NAT * 8; i += blockDim.x) atf[i] = 0.f;
    for (int c = t; c < np; c += blockDim.x) perm[c] = plan[20 + c];
    __syncthreads();
    for (int s = t; s < nsh; s += blockDim.x) {
        // shells are in packing order (s shells, then p shells, atom order
        // inside): an s shell right after an s shell of the same atom is its 2s
        const int g = md.sh0 + s, A = b.sh_atom[g];
        const int slot = b.sh_l[g] ? 2 : ((s > 0 && b.sh_atom[g - 1] == A && b.sh_l[g - 1] == 0) ? 1 : 0);
        // float4 offsets in the atom's entry: 1s a, c, -2ac at 0, 4, 8; 2s at
        // 12, 16, 20; 2p c, -2ac at 24, 28 (its exponents are the 2s ones)
        float *e = atx + A * TC_ATX;
        const int oa = slot == 0 ? 0 : 12, oc = slot == 0 ? 4 : (slot == 1 ? 16 : 24), om = oc + 4;
        for (int k = 0; k < 3; k++) {
            const double a = b.sh_ex[g * 3 + k], c = b.sh_co[g * 3 + k];
            if (slot < 2) e[oa + k] = (float)a;
            e[oc + k] = (float)c;
            e[om + k] = (float)(-2.0 * a * c);
        }
    }
    const double *D = b.mat + md.mat0 + (long long)M_D * n * n;
    if constexpr (FINAL) {
        float *Dp = (float *)(smem + C.L.D_hi);
        for (int i = t; i < np * np; i += blockDim.x) {
            const int pr = perm[i / np], pc = perm[i % np];
            Dp[i] = (pr >= 0 && pc >= 0) ? (float)D[pr * n + pc] : 0.f;
        }
    } else {
        for (int i = t; i < np * np / 4; i += blockDim.x) {
            const int row = i / (np / 4), kc = i % (np / 4);
            const int pr = perm[row];
            float v[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int pc = perm[kc * 4 + j];
                v[j] = (pr >= 0 && pc >= 0) ? (float)D[pr * n + pc] : 0.f;
            }
            float4 hi, lo;
            tc::split4(v, hi, lo);
            *(float4 *)(smem + C.L.D_hi + tc::coff(row, kc * 4, C.sg)) = hi;
            *(float4 *)(smem + C.L.D_lo + tc::coff(row, kc * 4, C.sg)) = lo;
        }
    }
    constexpr int U = NQ / 5;
    uint32_t uw[U > 0 ? U : 1];
#pragma unroll
    for (int k = 0; k < U; k++) uw[k] = (uint32_t)plan[C.q4 * 5 + k];
    const uint32_t rw = (uint32_t)plan[C.q4 * 5 + 4];
    if (C.warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&bar1)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&bar2)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    C.tT = tmem + TC_TCOL;
    C.tV = tmem + TC_VCOL;
    C.tS = tmem + TC_SCOL;
    C.lanes = (uint32_t)((C.warp & 3) * 32) << 16;  // this warp's TMEM lane quarter
    C.id = tc::idesc(128, np);
    C.id2 = tc::idesc(128, 2 * np);
    C.su = tc::smem_u32(smem);
    tc_loop<TA, FINAL, NQ>(b, C, uw, rw);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (C.warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

template <typename TA, bool FINAL, int NQ>
static void launch_tc_class(const DevBatch &b, int nchunk, int mode, const int *list, int count, cudaStream_t s) {
    const size_t sm = tc_layout(4 * NQ).total;
    cudaFuncSetAttribute(grid_xc_tc_kernel<TA, FINAL, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    grid_xc_tc_kernel<TA, FINAL, NQ><<<dim3(nchunk, count), TC_THREADS, sm, s>>>(b, nchunk, mode, list);
}

template <typename TA, bool FINAL>
static void launch_tc_all(const DevBatch &b, int nchunk, int mode, const TcClasses &cl, cudaStream_t s) {
    const int *l = cl.list;
    if (cl.count[0]) launch_tc_class<TA, FINAL, 4>(b, nchunk, mode, l + cl.off[0], cl.count[0], s);
    if (cl.count[1]) launch_tc_class<TA, FINAL, 8>(b, nchunk, mode, l + cl.off[1], cl.count[1], s);
    if (cl.count[2]) launch_tc_class<TA, FINAL, 12>(b, nchunk, mode, l + cl.off[2], cl.count[2], s);
    if (cl.count[3]) launch_tc_class<TA, FINAL, 16>(b, nchunk, mode, l + cl.off[3], cl.count[3], s);
    if (cl.count[4]) launch_tc_class<TA, FINAL, 20>(b, nchunk, mode, l + cl.off[4], cl.count[4], s);
}

void launch_grid_xc_tc(const DevBatch &b, int nchunk, int acc_fp64, int mode, const TcClasses &cl, cudaStream_t s) {
    if (acc_fp64) launch_tc_all<double, true>(b, nchunk, mode, cl, s);
    else launch_tc_all<float, false>(b, nchunk, mode, cl, s);
}

// ------------------------------------------------ bounded-wait self test
// The tensor-core kernels wait on mbarriers with an iteration limit; on
// expiry they set an error flag, drain, free tensor memory and return, and
// the host reports RKS_EDEVICE.  This kernel exercises that path without
// any fault: it waits on an mbarrier nothing will ever arrive at, with the
// given limit, and records whether the wait gave up.
__global__ void wait_selftest_kernel(int *gave_up, int spins) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t done = 0;
    for (int it = 0; it < spins && !done; it++) {
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(tc::smem_u32(&bar)), "r"(0u)
                     : "memory");
    }
    const bool ok = __syncthreads_and(done != 0);
    if (threadIdx.x == 0) *gave_up = ok ? 0 : 1;
}

void launch_wait_selftest(int *gave_up, int spins, cudaStream_t s) { wait_selftest_kernel<<<1, 32, 0, s>>>(gave_up, spins); }
