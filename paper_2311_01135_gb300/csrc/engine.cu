// Host engine and C ABI (include/rks.h): contexts, batches, the stage
// sequence of the SCF, results, profiling and the serving queue.
//
// Stage sequence of one batch (paper Section 3.1: iteration 0 precomputes
// V, T, S, I^2e and a first C; each iteration builds rho, V_xc, J, K and
// solves the eigenproblem):
//   setup: one-electron ints -> Schwarz Q -> kept pairs -> per-row quartet
//          counts -> row offsets -> packed ERIs -> grid -> H, E_nuc -> S^-1/2
//          and the core-Hamiltonian guess
//   iterate: zero accumulators -> J/K (packed store) -> grid XC -> FP64 step
//   final:   the same Fock build at the final precision -> plain diagonalisation
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/rks.h"
#include "common.cuh"
#include "kernels.h"

// ------------------------------------------------------------ errors
static thread_local std::string g_err;

int rks_cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    g_err = buf;
    return e == cudaErrorMemoryAllocation ? RKS_ENOMEM : RKS_ECUDA;
}

static int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

// ------------------------------------------------------------ STO-3G
// Hehre-Stewart-Pople STO-3G at the standard molecular exponents (H, C, N, O, F);
// 2s and 2p share exponents and are separate shells here.  Coefficients are for
// normalised primitives; the contracted functions are renormalised at start-up.
struct ShellDef {
    int l;
    double e[3], c[3];
};
struct ElemDef {
    int Z;
    int nsh;
    ShellDef sh[3];
};
static const double kC1s[3] = {0.15432897, 0.53532814, 0.44463454};
static const double kC2s[3] = {-0.09996723, 0.39951283, 0.70011547};
static const double kC2p[3] = {0.15591627, 0.60768372, 0.39195739};
static ElemDef g_elem[5] = {
    {1, 1, {{0, {3.42525091, 0.62391373, 0.16885540}, {0}}}},
    {6, 3, {{0, {71.6168370, 13.0450960, 3.5305122}, {0}}, {0, {2.9412494, 0.6834831, 0.2222899}, {0}},
            {1, {2.9412494, 0.6834831, 0.2222899}, {0}}}},
    {7, 3, {{0, {99.1061690, 18.0523120, 4.8856602}, {0}}, {0, {3.7804559, 0.8784966, 0.2857144}, {0}},
            {1, {3.7804559, 0.8784966, 0.2857144}, {0}}}},
    {8, 3, {{0, {130.7093200, 23.8088610, 6.4436083}, {0}}, {0, {5.0331513, 1.1695961, 0.3803890}, {0}},
            {1, {5.0331513, 1.1695961, 0.3803890}, {0}}}},
    {9, 3, {{0, {166.6791300, 30.3608120, 8.2168207}, {0}}, {0, {6.4648032, 1.5022812, 0.4885885}, {0}},
            {1, {6.4648032, 1.5022812, 0.4885885}, {0}}}},
};
static std::once_flag g_basis_once;

// Multiply the published coefficients by the primitive norms
// (2a/pi)^(3/4) (4a)^(l/2) and rescale to unit self-overlap.
static void init_basis() {
    for (auto &E : g_elem)
        for (int s = 0; s < E.nsh; s++) {
            ShellDef &sd = E.sh[s];
            const double *src = (E.Z == 1 || s == 0) ? kC1s : (sd.l == 0 ? kC2s : kC2p);
            double c[3];
            for (int k = 0; k < 3; k++)
                c[k] = src[k] * pow(2.0 * sd.e[k] / M_PI, 0.75) * pow(4.0 * sd.e[k], 0.5 * sd.l);
            double so = 0.0;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) {
                    double p = sd.e[i] + sd.e[j];
                    double v = pow(M_PI / p, 1.5);
                    if (sd.l == 1) v /= 2.0 * p;
                    so += c[i] * c[j] * v;
                }
            for (int k = 0; k < 3; k++) sd.c[k] = c[k] / sqrt(so);
        }
}

static const ElemDef *elem_of(int Z) {
    for (auto &E : g_elem)
        if (E.Z == Z) return &E;
    return nullptr;
}

extern "C" int rks_nbf(int32_t natom, const int32_t *Z) {
    if (natom <= 0 || !Z) return RKS_EINVAL;
    int n = 0;
    for (int i = 0; i < natom; i++) {
        const ElemDef *E = elem_of(Z[i]);
        if (!E) return RKS_EINVAL;
        for (int s = 0; s < E->nsh; s++) n += E->sh[s].l ? 3 : 1;
    }
    return n;
}

static int tc_plan_mol(int na, const int32_t *Zm, int nbf, int *plan);
static_assert(RKS_TC_PLAN == RKS_TC_PLAN_INTS, "one plan layout on both sides of the ABI");

extern "C" int rks_tc_plan(int32_t natom, const int32_t *Z, int32_t *plan) {
    std::call_once(g_basis_once, init_basis);
    if (!plan) return RKS_EINVAL;
    const int nbf = rks_nbf(natom, Z);
    if (nbf < 0) return nbf;
    return tc_plan_mol(natom, Z, nbf, plan);
}

extern "C" const char *rks_strerror(int code) {
    switch (code) {
    case RKS_OK: return "ok";
    case RKS_EINVAL: return "invalid argument";
    case RKS_ENOMEM: return "out of memory / over budget";
    case RKS_EAGAIN: return "queue full";
    case RKS_ENOTREADY: return "not ready";
    case RKS_ECUDA: return "CUDA error";
    case RKS_ETIMEOUT: return "timed out";
    case RKS_ENOTFOUND: return "unknown ticket";
    case RKS_EDEVICE: return "device-side check failed";
    default: return "unknown error";
    }
}

extern "C" int rks_options_default(rks_options *o) {
    if (!o) return RKS_EINVAL;
    memset(o, 0, sizeof *o);
    o->basis = 0;
    o->n_rad = 50;
    o->n_theta = 12;
    o->n_phi = 24;
    o->becke_iters = 3;
    o->precision = RKS_FP64;
    o->fixed_iters = 0;
    o->max_iters = 100;
    o->e_tol = 1e-9;
    o->err_tol = 1e-6;
    o->diis_space = 8;
    o->coords_in_angstrom = 0;
    o->xc = 1;
    o->max_slots = 4096;
    o->hbm_budget_bytes = 0;
    o->device = 0;
    o->use_graphs = 1;
    o->fix_theta = 0.1;
    o->grid_tc = 1;
    o->guess = RKS_GUESS_SAD;
    o->max_cohorts = 4;
    o->admit_wait_us = 20000;
    o->iter_precision = 0;
    o->recheck_err = 1e-4;
    o->recheck_fp64_err = 3e-4;
    return RKS_OK;
}

// --------------------------------------------------------- profiling
struct StageRec {
    std::string name;
    cudaEvent_t a, b;
    double units;
};

// ------------------------------------------------------------ context
struct rks_batch;
struct Ticket {
    int state = RKS_PENDING;
    int err = RKS_ECUDA;  // error rks_result reports for a failed ticket
    std::vector<int> Z;
    std::vector<double> xyz;
    rks_result_t res{};
    std::vector<double> eps, D;
    std::chrono::steady_clock::time_point t_submit;
};

struct rks_ctx {
    rks_options opt{};
    cudaStream_t stream = nullptr;
    double *boys64 = nullptr;
    float *boys32 = nullptr;
    double *rad = nullptr, *ang = nullptr;
    std::string err;
    // profiling
    bool prof = false;
    std::mutex prof_mu;
    std::vector<StageRec> recs;
    std::map<std::string, rks_stage_time> totals;
    // serving
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    size_t queue_cap = 1 << 20;
    size_t budget = 0;          // device bytes all cohorts in flight may hold
    // pinned host words for asynchronous readbacks, one per live batch
    int *pin = nullptr;
    std::vector<int> pin_free;
    int nsm = 152;              // multiprocessors of the device
};
static const int kPinSlots = 256;

extern "C" const char *rks_last_error(rks_ctx *ctx) {
    (void)ctx;
    return g_err.c_str();
}

extern "C" void *rks_stream(rks_ctx *ctx) { return ctx ? (void *)ctx->stream : nullptr; }

struct StageScope {
    rks_ctx *c;
    cudaStream_t st;
    StageRec r;
    bool on;
    StageScope(rks_ctx *ctx, cudaStream_t stream, const char *name, double units)
        : c(ctx), st(stream), on(ctx->prof) {
        if (on) {
            r.name = name;
            r.units = units;
            cudaEventCreate(&r.a);
            cudaEventCreate(&r.b);
            cudaEventRecord(r.a, st);
        }
    }
    ~StageScope() {
        if (on) {
            cudaEventRecord(r.b, st);
            std::lock_guard<std::mutex> lk(c->prof_mu);
            c->recs.push_back(r);
        }
    }
};

extern "C" int rks_profile_enable(rks_ctx *ctx, int32_t on) {
    if (!ctx) return RKS_EINVAL;
    ctx->prof = on != 0;
    return RKS_OK;
}

extern "C" int rks_profile_read(rks_ctx *ctx, rks_stage_time *out, int32_t cap) {
    if (!ctx) return RKS_EINVAL;
    CUDA_OK(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(ctx->prof_mu);
    for (auto &r : ctx->recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto &t = ctx->totals[r.name];
        snprintf(t.name, sizeof t.name, "%s", r.name.c_str());
        t.launches += 1;
        t.ms += ms;
        t.units += r.units;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    ctx->recs.clear();
    int n = 0;
    for (auto &kv : ctx->totals) {
        if (n < cap && out) out[n] = kv.second;
        n++;
    }
    ctx->totals.clear();
    return std::min(n, (int)cap);
}

// ------------------------------------------------------------- batch
struct HostMol {
    int natom, nbf, nocc, nsh, npair_all;
    long long eri_cap;
    int npts;
};

struct rks_batch {
    rks_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;  // the context stream, or a private one (serving cohorts)
    bool own_stream = false;
    size_t bytes = 0;               // device memory held
    int nmol = 0;
    int precision = 0;
    int max_nbf = 0, max_nsh = 0, max_atoms = 0, max_pair = 0;
    // molecules up to RKS_NBF_SMALL (shared-memory kernels) and above it
    // (global-memory kernels of large.cu): largest basis, shell and pair counts
    int max_nbf_small = 0, max_nsh_small = 0, max_pair_small = 0;
    int max_nbf_big = 0, max_nsh_big = 0, n_big = 0;
    bool direct = false;               // no packed store: J/K recompute the quartets every pass
    long long ncand = 0, nblk_total = 0;
    std::vector<HostMol> hm;
    std::vector<MolDesc> md;
    DevBatch d{};
    int *blk_mol = nullptr;
    std::vector<void *> allocs;
    bool set_up = false;
    double wall_s = 0.0;
    std::vector<MolState> st_host;
    bool st_valid = false;
    // one SCF iteration per iteration precision (RKS_ITER_* flags), captured
    // after one direct run of that launch sequence
    cudaGraphExec_t graph[4] = {};
    bool graph_warm[4] = {};
    bool graph_failed = false;
    int *recheck_d = nullptr;          // [2] molecules marked for the precise rerun / the FP64 redo
    int *recheck_list = nullptr;       // [nmol] indices marked for the FP64 redo
    int *recheck_list1 = nullptr;      // [nmol] indices marked for the precise rerun
    int n_precise = 0;                 // > 0 while the precise reruns are enqueued
    // inputs kept for the FP64 redo of unconverged molecules (coordinates in bohr)
    std::vector<int32_t> hZ, hnat;
    std::vector<double> hxyz;
    std::vector<long long> hatom0;
    TcClasses tcc{};                   // molecules of the tensor-core grid kernel by size class
    rks_batch *child = nullptr;        // FP64 batch of the molecules being redone
    int *child_map = nullptr;          // device: child molecule -> parent molecule
    cudaEvent_t child_done = nullptr;
    int pin_slot = -1;                 // ctx->pin words 2 pin_slot, 2 pin_slot + 1: readbacks (active
                                       // count; recheck counts)
    int *active_d = nullptr;
    int it_enq = 0;                    // SCF iterations enqueued so far
};

// The batch's two pinned host words for asynchronous readbacks.
static int *pinw(const rks_batch *b) { return b->ctx->pin + 2 * b->pin_slot; }

template <typename T> static int dalloc(rks_batch *b, T **p, size_t n) {
    void *q = nullptr;
    size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    // stream-ordered: no device-wide synchronisation when cohorts come and go
    cudaError_t e = cudaMallocAsync(&q, bytes, b->stream);
    if (e != cudaSuccess) return rks_cuda_fail(e, "cudaMallocAsync", __FILE__, __LINE__);
    b->allocs.push_back(q);
    b->bytes += bytes;
    *p = (T *)q;
    return RKS_OK;
}

static int validate(int natom, const int *Z, const double *xyz, int *nbf_out) {
    if (natom <= 0 || natom > 128 || !Z || !xyz) return fail(RKS_EINVAL, "natom out of range or null input");
    int nel = 0;
    for (int i = 0; i < natom; i++) {
        if (!elem_of(Z[i])) return fail(RKS_EINVAL, "unsupported element Z=" + std::to_string(Z[i]));
        nel += Z[i];
        for (int k = 0; k < 3; k++)
            if (!std::isfinite(xyz[3 * i + k])) return fail(RKS_EINVAL, "non-finite coordinate");
    }
    if (nel % 2) return fail(RKS_EINVAL, "odd electron count");
    int nbf = rks_nbf(natom, Z);
    if (nbf > RKS_NBF_CAP) return fail(RKS_EINVAL, "nbf " + std::to_string(nbf) + " above the compiled maximum");
    if (nbf_out) *nbf_out = nbf;
    return RKS_OK;
}

// Column plan of the tensor-core grid kernel for one molecule (layout in
// common.cuh).  Heavy atoms go round-robin to the quarters' units; hydrogens
// then fill the remaining unit slots and single columns, round-robin over the
// quarters with room.  Returns NQ, or 0 when no class fits (more than
// RKS_TC_NATMAX atoms, a basis above 80, or more heavy atoms than units): the
// CUDA-core kernel takes the molecule.
static int tc_plan_mol(int na, const int32_t *Zm, int nbf, int *plan) {
    if (na > RKS_TC_NATMAX) return 0;
    std::vector<int> heavy, light, ao_first(na);
    int ao = 0;
    for (int i = 0; i < na; i++) {
        const ElemDef *E = elem_of(Zm[i]);
        ao_first[i] = ao;
        if (E->nsh == 1 && E->sh[0].l == 0) {
            light.push_back(i);
            ao += 1;
        } else if (E->nsh == 3 && E->sh[0].l == 0 && E->sh[1].l == 0 && E->sh[2].l == 1 &&
                   E->sh[1].e[0] == E->sh[2].e[0] && E->sh[1].e[1] == E->sh[2].e[1] &&
                   E->sh[1].e[2] == E->sh[2].e[2]) {
            heavy.push_back(i);
            ao += 5;
        } else {
            return 0;
        }
    }
    for (int nq = 4; nq <= RKS_TC_NPMAX / 4; nq += 4) {
        if (4 * nq < nbf) continue;
        const int U = nq / 5, R = nq % 5;
        if ((int)heavy.size() > 4 * U) continue;
        // slots[q]: atom per column slot (unit k slot r at 5k + r, single column r at 5U + r)
        std::vector<std::vector<int>> slot(4, std::vector<int>(nq, RKS_TC_EMPTY));
        std::vector<int> hq(4, 0), used(4, 0);
        for (size_t i = 0; i < heavy.size(); i++) {
            const int q = (int)(i % 4), k = (int)(i / 4);
            slot[q][5 * k] = heavy[i];
            hq[q] = k + 1;
        }
        for (int q = 0; q < 4; q++) used[q] = 5 * hq[q];
        size_t li = 0;
        bool room = true;
        while (li < light.size() && room) {
            room = false;
            for (int q = 0; q < 4 && li < light.size(); q++)
                if (used[q] < nq) {
                    slot[q][used[q]++] = light[li++];
                    room = true;
                }
        }
        if (li < light.size()) continue;
        for (int q = 0; q < 4; q++) {
            for (int k = 0; k < 5; k++) plan[q * 5 + k] = 0;
            for (int k = 0; k < U; k++) {
                uint32_t w = 0;
                if (k < hq[q]) {
                    w = (1u << 31) | (uint32_t)slot[q][5 * k];
                    for (int r = 1; r < 5; r++) w |= (uint32_t)RKS_TC_EMPTY << (6 * r);
                } else {
                    for (int r = 0; r < 5; r++) w |= (uint32_t)slot[q][5 * k + r] << (6 * r);
                }
                plan[q * 5 + k] = (int)w;
            }
            uint32_t w = 0;
            for (int r = 0; r < 5; r++) w |= (uint32_t)(r < R ? slot[q][5 * U + r] : RKS_TC_EMPTY) << (6 * r);
            plan[q * 5 + 4] = (int)w;
            for (int j = 0; j < nq; j++) {
                const int c = q * nq + j, A = slot[q][j];
                int v = -1;
                if (j < 5 * U && j / 5 < hq[q]) v = ao_first[slot[q][5 * (j / 5)]] + j % 5;
                else if (A != RKS_TC_EMPTY) v = ao_first[A];
                plan[20 + c] = v;
            }
        }
        for (int c = 4 * nq; c < RKS_TC_NPMAX; c++) plan[20 + c] = -1;
        return nq;
    }
    return 0;
}

// Release the FP64 redo batch of the previous run.  Its results are read by
// the adopt kernel on the parent's stream, which may still be queued (a
// caller may enqueue the next run without waiting): drain the parent's
// stream before the child's memory goes.
static void child_free(rks_batch *b) {
    if (b->child) {
        cudaStreamSynchronize(b->stream);
        rks_batch_destroy(b->child);
    }
    b->child = nullptr;
    b->child_map = nullptr;
    if (b->child_done) cudaEventDestroy(b->child_done);
    b->child_done = nullptr;
}

extern "C" int rks_batch_destroy(rks_batch *b) {
    if (!b) return RKS_EINVAL;
    child_free(b);
    for (auto &gx : b->graph)
        if (gx) cudaGraphExecDestroy(gx);
    for (void *p : b->allocs) cudaFreeAsync(p, b->stream);
    cudaStreamSynchronize(b->stream);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    if (b->pin_slot >= 0) {
        std::lock_guard<std::mutex> lk(b->ctx->mu);
        b->ctx->pin_free.push_back(b->pin_slot);
    }
    delete b;
    return RKS_OK;
}

// Unscreened size of the packed store: candidate pairs in (l_P + l_Q, P, Q)
// order (s shells before p), row r holds n_r * sum_{s <= r} n_s elements.
static long long store_cap(int ns, int np) {
    long long cap = 0, pref = 0;
    const long long cnt[3] = {(long long)ns * (ns + 1) / 2, (long long)ns * np, (long long)np * (np + 1) / 2};
    const long long nr[3] = {1, 3, 9};
    for (int cls = 0; cls < 3; cls++)
        for (long long k = 0; k < cnt[cls]; k++) {
            pref += nr[cls];
            cap += nr[cls] * pref;
        }
    return cap;
}

// Device bytes one molecule adds to a batch (the allocations of
// batch_create_on, per molecule); the serving worker admits by this figure.
static size_t mol_bytes(const rks_options &o, int na, const int32_t *Z) {
    int ns = 0, np = 0, nbf = 0;
    for (int i = 0; i < na; i++) {
        const ElemDef *E = elem_of(Z[i]);
        if (!E) return 0;
        for (int k = 0; k < E->nsh; k++) {
            if (E->sh[k].l) np++; else ns++;
            nbf += E->sh[k].l ? 3 : 1;
        }
    }
    const size_t esz = o.precision ? 4 : 8;
    const long long nsh = ns + np, npair = nsh * (nsh + 1) / 2;
    const long long npts = (long long)na * o.n_rad * o.n_theta * o.n_phi;
    const long long nblk = (npts + RKS_PTS_BLOCK - 1) / RKS_PTS_BLOCK;
    const bool direct = o.direct_scf == RKS_DIRECT_ALWAYS;
    size_t b = sizeof(MolDesc) + sizeof(MolState) + 8 + (size_t)na * 28 + (size_t)nsh * 84;
    b += (size_t)npair * (8 + 4 + 8 + 8 + 8 + 4 + 8 + 45 * esz);
    if (o.precision == RKS_MIXED && (o.fix_theta > 0 || direct)) b += (size_t)npair * 45 * 8;
    if (o.precision == RKS_MIXED && o.fix_theta > 0 && !direct) b += 6 * (RKS_FIX_CAP * 16 + 4);
    if (!direct) b += (size_t)((store_cap(ns, np) + 3) & ~3LL) * esz;
    b += (size_t)nblk * RKS_PTS_BLOCK * 4 * esz + (size_t)nblk * 4;
    if (nbf > RKS_NBF_SMALL) b += (size_t)nblk * RKS_PTS_BLOCK * 4 * esz;  // X coefficients between the grid passes
    if (nbf > RKS_NBF_SMALL && o.precision == RKS_MIXED) b += (size_t)nbf * nbf * 3 * 4;  // FP32 copy of D
    if (o.precision == RKS_MIXED) b += (size_t)nblk * 16;  // grid block masks
    b += (size_t)nbf * nbf * (M_COUNT * 8 + 3 * 8);
    return b;
}

extern "C" int64_t rks_mol_bytes(const rks_options *options, int32_t natom, const int32_t *Z) {
    if (natom <= 0 || !Z) return fail(RKS_EINVAL, "natom <= 0 or null Z");
    std::call_once(g_basis_once, init_basis);
    rks_options o;
    if (options) o = *options; else rks_options_default(&o);
    const int nbf = rks_nbf(natom, Z);
    if (nbf < 0) return nbf;
    if (nbf > RKS_NBF_CAP) return fail(RKS_EINVAL, "nbf " + std::to_string(nbf) + " above the compiled maximum");
    return (int64_t)mol_bytes(o, natom, Z);
}

// precision: RKS_FP64 / RKS_MIXED, or -1 for the context's; bohr: coordinates
// are already in bohr (the FP64 redo of a batch's molecules).
static int batch_create_on(rks_ctx *ctx, cudaStream_t stream, bool own_stream, int32_t nmol, const int32_t *natom,
                           const int32_t *Z, const double *xyz, rks_batch **out, int precision = -1,
                           bool bohr = false) {
    if (!ctx || nmol <= 0 || !natom || !Z || !xyz || !out) {
        if (own_stream) cudaStreamDestroy(stream);
        return fail(RKS_EINVAL, "null argument");
    }
    std::call_once(g_basis_once, init_basis);
    rks_options o = ctx->opt;
    if (precision >= 0) o.precision = precision;
    const double conv = (o.coords_in_angstrom && !bohr) ? 1.0 / 0.52917721092 : 1.0;
    rks_batch *b = new rks_batch();
    b->ctx = ctx;
    b->stream = stream;
    b->own_stream = own_stream;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ctx->pin_free.empty()) {
            delete b;
            if (own_stream) cudaStreamDestroy(stream);
            return fail(RKS_ENOMEM, "too many live batches");
        }
        b->pin_slot = ctx->pin_free.back();
        ctx->pin_free.pop_back();
    }
    b->nmol = nmol;
    b->precision = o.precision;
    b->hm.resize(nmol);
    b->md.resize(nmol);
    const int nang = o.n_theta * o.n_phi, npa = o.n_rad * nang;
    // ---- host shell model
    std::vector<int> hZ, hsh_atom, hsh_l, hsh_ao0, hcand_mol;
    std::vector<double> haxyz, hsh_xyz, hsh_ex, hsh_co;
    std::vector<int2> hcand;
    std::vector<int> hblk_mol, hplan;
    long long atom_off = 0, sh_off = 0, pair_off = 0, pts_off = 0, eri_off = 0, mat_off = 0, acc_off = 0;
    for (int m = 0; m < nmol; m++) {
        const int na = natom[m];
        const int32_t *Zm = Z + atom_off;
        const double *Xm = xyz + 3 * atom_off;
        int nbf = 0;
        int rc = validate(na, Zm, Xm, &nbf);
        if (rc) {
            delete b;
            return fail(rc, "molecule " + std::to_string(m) + ": " + g_err);
        }
        int nel = 0;
        for (int i = 0; i < na; i++) nel += Zm[i];
        // shells in AO order, then reorder: s first, then p (stable)
        struct Sh { int atom, l, ao0; const ShellDef *sd; };
        std::vector<Sh> ao;
        int aoi = 0;
        for (int i = 0; i < na; i++) {
            const ElemDef *E = elem_of(Zm[i]);
            for (int s = 0; s < E->nsh; s++) {
                ao.push_back({i, E->sh[s].l, aoi, &E->sh[s]});
                aoi += E->sh[s].l ? 3 : 1;
            }
        }
        std::vector<Sh> sh;
        for (int l = 0; l <= 1; l++)
            for (auto &x : ao)
                if (x.l == l) sh.push_back(x);
        const int nsh = (int)sh.size();
        for (auto &x : sh) {
            hsh_atom.push_back(x.atom);
            hsh_l.push_back(x.l);
            hsh_ao0.push_back(x.ao0);
            for (int k = 0; k < 3; k++) {
                hsh_xyz.push_back(Xm[3 * x.atom + k] * conv);
                hsh_ex.push_back(x.sd->e[k]);
                hsh_co.push_back(x.sd->c[k]);
            }
        }
        b->hatom0.push_back((long long)hZ.size());
        b->hnat.push_back(na);
        for (int i = 0; i < na; i++) {
            hZ.push_back(Zm[i]);
            for (int k = 0; k < 3; k++) haxyz.push_back(Xm[3 * i + k] * conv);
        }
        // candidate pairs ordered by (l_P + l_Q, P, Q)
        std::vector<int2> pr;
        for (int cls = 0; cls <= 2; cls++)
            for (int P = 0; P < nsh; P++)
                for (int Q = 0; Q <= P; Q++)
                    if (sh[P].l + sh[Q].l == cls) pr.push_back(make_int2(P, Q));
        const int npair_all = (int)pr.size();
        int ns = 0;
        for (auto &x : sh) ns += x.l == 0;
        const long long cap = store_cap(ns, nsh - ns);
        for (auto &p : pr) {
            hcand.push_back(p);
            hcand_mol.push_back(m);
        }
        const int npts = na * npa;
        const int nblk = (npts + RKS_PTS_BLOCK - 1) / RKS_PTS_BLOCK;
        for (int k = 0; k < nblk; k++) hblk_mol.push_back(m);
        MolDesc &d = b->md[m];
        d.natom = na; d.nbf = nbf; d.nocc = nel / 2; d.nsh = nsh;
        d.atom0 = (int)atom_off; d.sh0 = (int)sh_off; d.npair_all = npair_all; d.pair0 = (int)pair_off;
        d.npts = npts; d.nblk = nblk; d.pts0 = pts_off;
        d.eri0 = eri_off; d.eri_cap = cap;
        d.mat0 = mat_off; d.acc0 = acc_off;
        if (o.precision == RKS_MIXED) {
            int pl[RKS_TC_PLAN];
            d.tcq = tc_plan_mol(na, Zm, nbf, pl);
            hplan.insert(hplan.end(), pl, pl + RKS_TC_PLAN);
        }
        d.big = nbf > RKS_NBF_SMALL;
        b->hm[m] = {na, nbf, nel / 2, nsh, npair_all, cap, npts};
        b->max_nbf = std::max(b->max_nbf, nbf);
        b->max_nsh = std::max(b->max_nsh, nsh);
        b->max_pair = std::max(b->max_pair, npair_all);
        b->max_atoms = std::max(b->max_atoms, na);
        if (d.big) {
            b->n_big++;
            b->max_nbf_big = std::max(b->max_nbf_big, nbf);
            b->max_nsh_big = std::max(b->max_nsh_big, nsh);
        } else {
            b->max_nbf_small = std::max(b->max_nbf_small, nbf);
            b->max_nsh_small = std::max(b->max_nsh_small, nsh);
            b->max_pair_small = std::max(b->max_pair_small, npair_all);
        }
        atom_off += na;
        sh_off += nsh;
        pair_off += npair_all;
        pts_off += (long long)nblk * RKS_PTS_BLOCK;
        eri_off += (cap + 3) & ~3LL;  // keep every molecule's store 16-byte aligned
        mat_off += (long long)M_COUNT * nbf * nbf;
        acc_off += 3LL * nbf * nbf;
    }
    b->ncand = pair_off;
    b->nblk_total = pts_off / RKS_PTS_BLOCK;
    // ---- device buffers
    DevBatch &d = b->d;
    d.nmol = nmol;
    d.precision = o.precision;
    d.xc = o.xc;
    d.a0 = o.xc ? 0.2 : 1.0;
    d.n_rad = o.n_rad; d.n_theta = o.n_theta; d.n_phi = o.n_phi; d.becke_iters = o.becke_iters;
    d.diis_space = std::max(1, std::min(o.diis_space, RKS_DIIS_MAX));
    d.fixed_iters = o.fixed_iters;
    d.max_iters = o.max_iters;
    d.guess = o.guess;
    d.e_tol = o.e_tol;
    d.err_tol = o.err_tol;
    d.recheck_err = o.recheck_err;
    d.recheck_fp64_err = o.recheck_fp64_err;
    d.boys64 = ctx->boys64;
    d.boys32 = ctx->boys32;
    const size_t esz = o.precision ? sizeof(float) : sizeof(double);
    // direct SCF: always, or (auto) when the packed stores would take more
    // than 70% of the device memory free now
    b->direct = o.direct_scf == RKS_DIRECT_ALWAYS;
    if (o.direct_scf == RKS_DIRECT_AUTO) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) b->direct = (double)eri_off * esz > 0.7 * (double)fr;
    }
    d.direct = b->direct ? 1 : 0;
    const bool want64 = o.precision == RKS_MIXED && (o.fix_theta > 0 || b->direct);  // FP64 pair data
    const bool want_fix = o.precision == RKS_MIXED && o.fix_theta > 0 && !b->direct;   // FP64 recompute lists
    int rc = 0;
    void *gcf = nullptr, *gdt = nullptr;
    MolDesc *dmol; MolState *dst; int *dZ, *dsa, *dsl, *dsao, *dcm, *dnp, *drnq; double *dax, *dsx, *dse, *dsc, *dcq, *dkq;
    int2 *dcand, *dkp; long long *droff; void *store; void *gx, *gy, *gz, *gw; double *mat, *accd;
    void *pairprim, *pairprim64 = nullptr;
    int4 *fixlist = nullptr;
    int *fixcount = nullptr;
    if ((rc = dalloc(b, &dmol, nmol)) || (rc = dalloc(b, &dst, nmol)) || (rc = dalloc(b, &dZ, atom_off)) ||
        (rc = dalloc(b, &dax, 3 * atom_off)) || (rc = dalloc(b, &dsa, sh_off)) || (rc = dalloc(b, &dsl, sh_off)) ||
        (rc = dalloc(b, &dsao, sh_off)) || (rc = dalloc(b, &dsx, 3 * sh_off)) || (rc = dalloc(b, &dse, 3 * sh_off)) ||
        (rc = dalloc(b, &dsc, 3 * sh_off)) || (rc = dalloc(b, &dcand, pair_off)) || (rc = dalloc(b, &dcm, pair_off)) ||
        (rc = dalloc(b, &dcq, pair_off)) || (rc = dalloc(b, &dkp, pair_off)) || (rc = dalloc(b, &dkq, pair_off)) ||
        (rc = dalloc(b, &dnp, nmol)) || (rc = dalloc(b, &drnq, pair_off)) || (rc = dalloc(b, &droff, pair_off + nmol)) ||
        (rc = dalloc(b, (unsigned char **)&store, (b->direct ? 4 : eri_off) * esz)) ||
        (rc = dalloc(b, (unsigned char **)&pairprim, pair_off * 9 * 5 * esz)) ||
        (want64 && (rc = dalloc(b, (unsigned char **)&pairprim64, pair_off * 9 * 5 * sizeof(double)))) ||
        (want_fix && ((rc = dalloc(b, &fixlist, (size_t)nmol * 6 * RKS_FIX_CAP)) ||
                      (rc = dalloc(b, &fixcount, (size_t)nmol * 6)))) ||
        (b->n_big > 0 && (rc = dalloc(b, (unsigned char **)&gcf, pts_off * 4 * esz))) ||
        (b->n_big > 0 && o.precision == RKS_MIXED && (rc = dalloc(b, (float **)&gdt, acc_off))) ||
        (rc = dalloc(b, (unsigned char **)&gx, pts_off * esz)) || (rc = dalloc(b, (unsigned char **)&gy, pts_off * esz)) ||
        (rc = dalloc(b, (unsigned char **)&gz, pts_off * esz)) || (rc = dalloc(b, (unsigned char **)&gw, pts_off * esz)) ||
        (rc = dalloc(b, &mat, mat_off)) || (rc = dalloc(b, &accd, acc_off)) ||
        (rc = dalloc(b, &b->blk_mol, b->nblk_total)) || (rc = dalloc(b, &b->active_d, 1)) ||
        (rc = dalloc(b, &b->recheck_d, 2)) || (rc = dalloc(b, &b->recheck_list, nmol)) ||
        (rc = dalloc(b, &b->recheck_list1, nmol)) ||
        (o.precision == RKS_MIXED && (rc = dalloc(b, &d.blk_mask, 2 * b->nblk_total))) ||
        (o.precision == RKS_MIXED && (rc = dalloc(b, (int **)&b->tcc.list, nmol))) ||
        (o.precision == RKS_MIXED && (rc = dalloc(b, (int **)&d.tc_plan, (size_t)nmol * RKS_TC_PLAN))) ||
        (rc = dalloc(b, &d.jk_next, nmol))) {
        rks_batch_destroy(b);
        return rc;
    }
    d.mol = dmol; d.st = dst; d.Z = dZ; d.axyz = dax; d.sh_atom = dsa; d.sh_l = dsl; d.sh_ao0 = dsao;
    d.sh_xyz = dsx; d.sh_ex = dse; d.sh_co = dsc; d.cand = dcand; d.cand_mol = dcm; d.cand_q = dcq;
    d.kpair = dkp; d.kq = dkq; d.npair = dnp; d.row_nq = drnq; d.row_off = droff; d.store = store;
    d.pairprim = pairprim;
    d.pairprim64 = pairprim64;
    d.fixlist = fixlist;
    d.fixcount = fixcount;
    d.fix_theta = o.fix_theta;
    d.gx = gx; d.gy = gy; d.gz = gz; d.gw = gw; d.mat = mat; d.accd = accd; d.accx = (Fx *)accd;  // one buffer, two views
    d.gcf = gcf;
    d.gdt = gdt;
    cudaStream_t s = b->stream;
#define UP(dst_, src_)                                                                                      \
    if (!(src_).empty()) {                                                                                  \
        cudaError_t e_ = cudaMemcpyAsync(dst_, (src_).data(), (src_).size() * sizeof((src_)[0]),          \
                                         cudaMemcpyHostToDevice, s);                                        \
        if (e_ != cudaSuccess) { rks_batch_destroy(b); return rks_cuda_fail(e_, "H2D", __FILE__, __LINE__); } \
    }
    UP(dmol, b->md);
    UP(dZ, hZ);
    UP(dax, haxyz);
    UP(dsa, hsh_atom);
    UP(dsl, hsh_l);
    UP(dsao, hsh_ao0);
    UP(dsx, hsh_xyz);
    UP(dse, hsh_ex);
    UP(dsc, hsh_co);
    UP(dcand, hcand);
    UP(dcm, hcand_mol);
    UP(b->blk_mol, hblk_mol);
    if (b->tcc.list) {
        // tensor-core grid kernel: molecules by column class NQ = 4 (k + 1)
        std::vector<int> lst;
        for (int k = 0; k < 5; k++) {
            b->tcc.off[k] = (int)lst.size();
            for (int m = 0; m < nmol; m++)
                if (b->md[m].tcq == 4 * (k + 1)) lst.push_back(m);
            b->tcc.count[k] = (int)lst.size() - b->tcc.off[k];
        }
        UP((int *)b->tcc.list, lst);
        UP((int *)d.tc_plan, hplan);
    }
#undef UP
    b->hZ = hZ;
    b->hxyz = haxyz;
    cudaError_t e = cudaMemsetAsync(dst, 0, sizeof(MolState) * nmol, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mat, 0, sizeof(double) * mat_off, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        rks_batch_destroy(b);
        return rks_cuda_fail(e, "batch upload", __FILE__, __LINE__);
    }
    *out = b;
    return RKS_OK;
}

extern "C" int rks_batch_create(rks_ctx *ctx, int32_t nmol, const int32_t *natom, const int32_t *Z,
                                const double *xyz, rks_batch **out) {
    if (!ctx) return fail(RKS_EINVAL, "null context");
    return batch_create_on(ctx, ctx->stream, false, nmol, natom, Z, xyz, out);
}

// -------------------------------------------------------------- stages
static int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rks_cuda_fail(e, what, __FILE__, __LINE__);
    return RKS_OK;
}

extern "C" int rks_batch_setup(rks_batch *b) {
    if (!b) return RKS_EINVAL;
    rks_ctx *c = b->ctx;
    cudaStream_t s = b->stream;
    const DevBatch &d = b->d;
    const int fp32 = b->precision;
    { StageScope sc(c, s, "onee", 0); launch_onee(d, (int)b->ncand, s); }
    { StageScope sc(c, s, "schwarz", 0); launch_schwarz(d, (int)b->ncand, s); }
    { StageScope sc(c, s, "pairs", 0); launch_compact_pairs(d, s); }
    { StageScope sc(c, s, "row_count", 0); launch_row_count(d, (int)b->ncand, s); }
    { StageScope sc(c, s, "row_scan", 0); launch_row_scan(d, s); }
    { StageScope sc(c, s, "pair_prim", 0); launch_pair_prim(d, (int)b->ncand, fp32, s); }
    if (!b->direct) { StageScope sc(c, s, "eri", 0); launch_eri_store(d, (int)b->ncand, fp32, s); }
    if (d.fixlist) { StageScope sc(c, s, "fix_list", 0); launch_fix_list(d, s); }
    { StageScope sc(c, s, "grid_build", 0); launch_grid_build(d, b->nblk_total, b->blk_mol, c->rad, c->ang, b->max_atoms, s); }
    { StageScope sc(c, s, "grid_masks", 0); launch_grid_masks(d, b->nblk_total, b->blk_mol, s); }
    { StageScope sc(c, s, "scf_init", 0); launch_scf_init(d, s); }
    { StageScope sc(c, s, "scf_guess", 0); launch_scf_guess(d, b->max_nbf_small, 0, s); }
    int rc = check_launch("setup kernels");
    if (rc) return rc;
    b->it_enq = 0;
    b->set_up = true;
    b->st_valid = false;
    return RKS_OK;
}

// One Fock build for every (active when mode 0) molecule.  prec: RKS_ITER_*
// flags; on the mixed path RKS_ITER_JK_FINAL forms the J/K products in FP64
// and adds the FP64 recompute of the largest quartets, RKS_ITER_GRID_FINAL
// forms the density on the CUDA cores (the final step uses both).
static int fock_pass(rks_batch *b, int prec, int mode) {
    rks_ctx *c = b->ctx;
    cudaStream_t s = b->stream;
    const DevBatch &d = b->d;
    long long acc_elems = 0;
    for (auto &m : b->md) acc_elems += 3LL * m.nbf * m.nbf;
    CUDA_OK(cudaMemsetAsync(d.accd, 0, sizeof(double) * acc_elems, s));  // zero in both views
    launch_reset_exc(d, s);
    // blocks per molecule; J/K rows are shared out dynamically.  Defaults from
    // the autotuner (tune.py) on the 9-11-heavy-atom workload.
    // Thread blocks per molecule.  J/K sums in exact fixed point (mixed) or
    // FP64 (FP64 path), so its block count only spreads small batches over
    // the GPU (at least two blocks per multiprocessor).  The mixed grid
    // kernels keep 16 per molecule, so that a molecule sums its points in the
    // same groups in any batch; the FP64 path's grid sums reorder at ~1e-16
    // and spread like J/K.  Defaults from the autotuner (tune.py) on the
    // 9-11-heavy-atom workload.
    const int spread = (2 * c->nsm + b->nmol - 1) / b->nmol;
    const int nchunk_jk = c->opt.jk_chunks > 0 ? c->opt.jk_chunks : std::min(256, std::max(8, spread));
    CUDA_OK(cudaMemsetAsync(d.jk_next, 0, sizeof(int) * b->nmol, s));
    const int jk_fin = b->precision == 0 || (prec & RKS_ITER_JK_FINAL);
    const int gr_fin = b->precision == 0 || (prec & RKS_ITER_GRID_FINAL);
    const char *jk_name = mode ? "jk_final" : (jk_fin ? "jk_precise" : "jk");
    if (!b->direct && b->max_nbf_small > 0) {
        StageScope sc(c, s, jk_name, 0);
        if (launch_jk(d, nchunk_jk, jk_fin, mode, b->max_nbf_small, b->max_pair_small, s))
            return fail(RKS_EINVAL, "basis too large for the J/K kernel's shared memory");
    }
    if (b->direct || b->n_big > 0) {
        // molecules above RKS_NBF_SMALL, or every molecule in direct SCF
        const char *nm = b->direct ? (mode ? "jk_direct_final" : "jk_direct") : (mode ? "jk_large_final" : "jk_large");
        StageScope sc(c, s, nm, 0);
        const int nm_mol = b->direct ? b->nmol : b->n_big;
        const int nch = c->opt.jk_chunks > 0 ? c->opt.jk_chunks
                                             : std::min(256, std::max(8, (4 * c->nsm + nm_mol - 1) / nm_mol));
        if (launch_jk_large(d, nch, jk_fin, mode, b->direct ? 1 : 0, s))
            return fail(RKS_EINVAL, "direct SCF final step without FP64 pair data");
    }
    if (jk_fin && b->precision == RKS_MIXED && d.fixlist) {
        StageScope sc(c, s, mode ? "jk_fp64_fix" : "jk_fp64_fix_it", 0);
        if (mode == 0 && b->n_precise > 0) {
            // the precise reruns: only their molecules, spread over the GPU
            const int nch = std::min(256, std::max(8, (8 * c->nsm + b->n_precise - 1) / b->n_precise));
            launch_jk_fix(d, mode, s, b->recheck_list1, b->n_precise, nch);
        } else {
            launch_jk_fix(d, mode, s);
        }
    }
    if (d.xc) {
        // Molecules with a tensor-core column plan (MolDesc::tcq, decided per
        // molecule, never per batch) run that kernel; in the final step it forms the
        // density on the CUDA cores (the tensor cores' truncating accumulation
        // would bias E_xc).  The others run the CUDA-core kernel.
        const bool tc = b->precision == RKS_MIXED && c->opt.grid_tc;
        bool need_cc = !tc;
        if (tc) {
            bool any_tc = false;
            for (auto &m : b->md) {
                if (m.tcq) any_tc = true;
                else if (!m.big) need_cc = true;
            }
            if (any_tc) {
                const int nchunk_tc = c->opt.grid_chunks > 0 ? c->opt.grid_chunks : 16;
                StageScope sc(c, s, mode ? "grid_xc_tc_final" : (gr_fin ? "grid_xc_tc_precise" : "grid_xc_tc"), 0);
                launch_grid_xc_tc(d, nchunk_tc, gr_fin, mode, b->tcc, s);
            }
        }
        if (need_cc && b->max_nbf_small > 0) {
            const int nchunk_gx = c->opt.grid_chunks > 0 ? c->opt.grid_chunks
                                  : (b->precision == RKS_FP64 ? std::min(256, std::max(16, spread)) : 16);
            StageScope sc(c, s, mode ? "grid_xc_final" : (gr_fin ? "grid_xc_precise" : "grid_xc"), 0);
            launch_grid_xc(d, nchunk_gx, gr_fin, mode, tc ? 1 : 0, b->max_nbf_small, b->max_nsh_small, s);
        }
        if (b->n_big > 0) {
            // molecules above RKS_NBF_SMALL: two passes, global-memory D and V'.
            // The mixed path keeps 64 blocks per molecule, so that a molecule
            // sums its points in the same groups in any batch; FP64 spreads.
            const int nchunk_lg = c->opt.grid_chunks > 0 ? c->opt.grid_chunks
                                  : b->precision == RKS_MIXED
                                      ? 64
                                      : std::min(512, std::max(16, (2 * c->nsm + b->n_big - 1) / b->n_big));
            StageScope sc(c, s, mode ? "grid_large_final" : (gr_fin ? "grid_large_precise" : "grid_large"), 0);
            if (launch_grid_xc_large(d, nchunk_lg, gr_fin, mode, b->max_nbf_big, b->max_nsh_big, s))
                return fail(RKS_EINVAL, "basis too large for the grid kernels' shared memory");
        }
    }
    return check_launch("fock pass");
}

// One SCF iteration for every molecule still iterating: Fock build and the
// per-molecule step (DIIS, diagonalisation, density, convergence flags).
static int enqueue_one_iter(rks_batch *b, int prec) {
    int rc = fock_pass(b, prec, 0);
    if (rc) return rc;
    StageScope sc(b->ctx, b->stream, "scf_step", 0);
    launch_scf_step(b->d, b->precision == 0, b->max_nbf_small, b->stream);
    return check_launch("scf step");
}

// Enqueue n iterations at iteration precision prec.  The iteration is the
// same launch sequence every time (inactive molecules are skipped by the
// kernels, not by the host), so after one direct run it is captured once as a
// CUDA graph and replayed; stage profiling needs per-launch events and turns
// the graph off.
static int enqueue_iters(rks_batch *b, int n, int prec) {
    rks_ctx *c = b->ctx;
    cudaStream_t s = b->stream;
    int rc;
    prec &= 3;
    for (int k = 0; k < n; k++, b->it_enq++) {
        const bool use_graph = c->opt.use_graphs && !c->prof && !b->graph_failed && b->graph_warm[prec] &&
                               b->n_precise == 0;
        cudaGraphExec_t &gx = b->graph[prec];
        if (use_graph && !gx) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                rc = enqueue_one_iter(b, prec);
                e = cudaStreamEndCapture(s, &g);
                if (e == cudaSuccess && rc == RKS_OK) e = cudaGraphInstantiate(&gx, g, 0);
                if (g) cudaGraphDestroy(g);
            }
            if (e != cudaSuccess || !gx) {
                // capture is an optimisation: fall back to direct launches
                cudaGetLastError();
                gx = nullptr;
                b->graph_failed = true;
            }
        }
        if (gx && use_graph) {
            CUDA_OK(cudaGraphLaunch(gx, s));
        } else {
            if ((rc = enqueue_one_iter(b, prec))) return rc;
            b->graph_warm[prec] = true;
        }
    }
    return RKS_OK;
}

// Iteration precision of the first pass: the option on the mixed path.
static int iter_prec(const rks_batch *b) { return b->precision == RKS_MIXED ? (b->ctx->opt.iter_precision & 3) : 0; }
static const int kPrecise = RKS_ITER_JK_FINAL | RKS_ITER_GRID_FINAL;

static bool recheck_on(const rks_batch *b) {
    return b->precision == RKS_MIXED && b->d.fixed_iters > 0 && (b->d.recheck_err > 0.0 || b->d.recheck_fp64_err > 0.0);
}

// Mark the molecules to run again (precise rerun, started from the initial
// guess here) or to redo in FP64; the two counts go to the batch's pinned
// words, the FP64 list to recheck_list.
static int enqueue_recheck_start(rks_batch *b) {
    cudaStream_t s = b->stream;
    {
        StageScope sc(b->ctx, s, "recheck_mark", 0);
        launch_mark_recheck(b->d, b->recheck_d, b->recheck_list, b->recheck_list1, s);
    }
    {
        StageScope sc(b->ctx, s, "scf_guess", 0);
        launch_scf_guess(b->d, b->max_nbf_small, 1, s);
    }
    CUDA_OK(cudaMemcpyAsync(pinw(b), b->recheck_d, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    return check_launch("recheck start");
}

// Start the FP64 redo of the n molecules in recheck_list (host-visible once
// the marking has completed): a child batch on its own stream, whose work
// overlaps the parent's precise rerun and final step.
static int start_fp64_redo(rks_batch *b, int n) {
    std::vector<int> list(n);
    CUDA_OK(cudaMemcpy(list.data(), b->recheck_list, sizeof(int) * n, cudaMemcpyDeviceToHost));
    std::sort(list.begin(), list.end());
    std::vector<int32_t> na, Z;
    std::vector<double> xyz;
    for (int m : list) {
        na.push_back(b->hnat[m]);
        Z.insert(Z.end(), b->hZ.begin() + b->hatom0[m], b->hZ.begin() + b->hatom0[m] + b->hnat[m]);
        xyz.insert(xyz.end(), b->hxyz.begin() + 3 * b->hatom0[m], b->hxyz.begin() + 3 * (b->hatom0[m] + b->hnat[m]));
    }
    cudaStream_t cs = nullptr;
    CUDA_OK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    int rc = batch_create_on(b->ctx, cs, true, n, na.data(), Z.data(), xyz.data(), &b->child, RKS_FP64, true);
    if (rc) return rc;
    if ((rc = dalloc(b->child, &b->child_map, n))) return rc;
    CUDA_OK(cudaMemcpyAsync(b->child_map, list.data(), sizeof(int) * n, cudaMemcpyHostToDevice, cs));
    if ((rc = rks_batch_run(b->child))) return rc;
    CUDA_OK(cudaEventCreateWithFlags(&b->child_done, cudaEventDisableTiming));
    CUDA_OK(cudaEventRecord(b->child_done, cs));
    return RKS_OK;
}

// After the parent's final step: wait for the FP64 redo and take its results.
static int enqueue_adopt(rks_batch *b) {
    if (!b->child) return RKS_OK;
    CUDA_OK(cudaStreamWaitEvent(b->stream, b->child_done, 0));
    StageScope sc(b->ctx, b->stream, "recheck_adopt", 0);
    launch_adopt(b->d, b->child->d, b->child_map, b->child->nmol, b->stream);
    return check_launch("adopt");
}

// Count of molecules still iterating, copied to the batch's pinned word.
static int enqueue_active_count(rks_batch *b) {
    launch_count_active(b->d, b->active_d, b->stream);
    CUDA_OK(cudaMemcpyAsync(pinw(b), b->active_d, sizeof(int), cudaMemcpyDeviceToHost,
                            b->stream));
    return check_launch("count active");
}

// Final step: every molecule, FP64 accumulation.
static int enqueue_final(rks_batch *b) {
    int rc = fock_pass(b, kPrecise, 1);
    if (rc) return rc;
    StageScope sc(b->ctx, b->stream, "scf_final", 0);
    launch_scf_final(b->d, 1, b->max_nbf_small, b->stream);
    b->st_valid = false;
    return check_launch("final");
}

static const int kCheckEvery = 4;

extern "C" int rks_batch_run(rks_batch *b) {
    if (!b) return RKS_EINVAL;
    auto t0 = std::chrono::steady_clock::now();
    int rc;
    if (!b->set_up && (rc = rks_batch_setup(b))) return rc;
    const DevBatch &d = b->d;
    const int prec = iter_prec(b);
    child_free(b);
    if (d.fixed_iters > 0) {
        if ((rc = enqueue_iters(b, d.fixed_iters, prec))) return rc;
        if (recheck_on(b)) {
            if ((rc = enqueue_recheck_start(b))) return rc;
            CUDA_OK(cudaStreamSynchronize(b->stream));
            const int n_precise = pinw(b)[0], n_fp64 = pinw(b)[1];
            if (n_fp64 > 0 && (rc = start_fp64_redo(b, n_fp64))) return rc;
            b->n_precise = n_precise;
            if (n_precise > 0) rc = enqueue_iters(b, d.fixed_iters, kPrecise);
            b->n_precise = 0;
            if (rc) return rc;
        }
    } else {
        while (b->it_enq < d.max_iters) {
            if ((rc = enqueue_iters(b, std::min(kCheckEvery, d.max_iters - b->it_enq), prec))) return rc;
            if ((rc = enqueue_active_count(b))) return rc;
            CUDA_OK(cudaStreamSynchronize(b->stream));
            if (pinw(b)[0] == 0) break;
        }
    }
    if ((rc = enqueue_final(b))) return rc;
    if ((rc = enqueue_adopt(b))) return rc;
    b->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return RKS_OK;
}

extern "C" int rks_batch_sync(rks_batch *b) {
    if (!b) return RKS_EINVAL;
    b->st_host.resize(b->nmol);
    CUDA_OK(cudaMemcpyAsync(b->st_host.data(), b->d.st, sizeof(MolState) * b->nmol, cudaMemcpyDeviceToHost,
                            b->stream));
    CUDA_OK(cudaStreamSynchronize(b->stream));
    b->st_valid = true;
    for (auto &st : b->st_host)
        if (st.err_flag) return fail(RKS_EDEVICE, "device-side consistency flag set");
    return RKS_OK;
}

extern "C" int rks_batch_fock(rks_batch *b, const double *D_all, int32_t final_step) {
    if (!b || !D_all) return RKS_EINVAL;
    int rc;
    if (!b->set_up && (rc = rks_batch_setup(b))) return rc;
    long long off = 0;
    for (int m = 0; m < b->nmol; m++) {
        const MolDesc &md = b->md[m];
        long long nn = (long long)md.nbf * md.nbf;
        CUDA_OK(cudaMemcpyAsync(b->d.mat + md.mat0 + (long long)M_D * nn, D_all + off, nn * sizeof(double),
                                cudaMemcpyHostToDevice, b->stream));
        off += nn;
    }
    const int acc64 = final_step || b->precision == 0;
    if ((rc = fock_pass(b, final_step ? kPrecise : iter_prec(b), 1))) return rc;
    launch_fock_only(b->d, acc64, b->stream);
    b->st_valid = false;
    return check_launch("fock only");
}

static int ensure_state(rks_batch *b) {
    if (b->st_valid) return RKS_OK;
    return rks_batch_sync(b);
}

static double paper_std(const MolState &st) {
    int n = std::min(st.iter, 5);
    if (n < 5) return 1e30;
    double mean = 0, v = 0;
    for (int k = st.iter - 5; k < st.iter; k++) mean += st.Ehist[k % RKS_NHIST];
    mean /= 5;
    for (int k = st.iter - 5; k < st.iter; k++) v += pow(st.Ehist[k % RKS_NHIST] - mean, 2);
    return sqrt(v / 5);
}

extern "C" int rks_batch_result(rks_batch *b, int32_t m, rks_result_t *out, double *eps_out, double *D_out,
                                int32_t cap_nbf) {
    if (!b || m < 0 || m >= b->nmol || !out) return RKS_EINVAL;
    int rc = ensure_state(b);
    if (rc && rc != RKS_EDEVICE) return rc;
    const MolState &st = b->st_host[m];
    const MolDesc &md = b->md[m];
    if ((eps_out || D_out) && cap_nbf < md.nbf) return fail(RKS_EINVAL, "cap_nbf smaller than nbf");
    memset(out, 0, sizeof *out);
    out->status = st.status;
    if (b->d.fixed_iters == 0 && !st.converged && st.status == RKS_STATUS_OK) out->status = RKS_STATUS_NOT_CONVERGED;
    out->nbf = md.nbf;
    out->n_occ = md.nocc;
    out->iters = st.iter;
    out->e_total = st.E;
    out->e_homo = st.eps_homo;
    out->e_lumo = st.eps_lumo;
    out->gap = st.eps_lumo - st.eps_homo;
    out->e_xc = st.Exc;
    out->e_nuc = st.Enuc;
    out->latency_s = b->wall_s;
    out->paper_converged = paper_std(st) < 0.01;
    out->rechecked = st.rechecked;
    out->err_max = st.max_err;
    out->de_last = st.iter >= 2 ? fabs(st.Ehist[(st.iter - 1) % RKS_NHIST] - st.Ehist[(st.iter - 2) % RKS_NHIST]) : 0.0;
    if (eps_out) memcpy(eps_out, st.eps, sizeof(double) * md.nbf);
    if (D_out) {
        long long nn = (long long)md.nbf * md.nbf;
        CUDA_OK(cudaMemcpyAsync(D_out, b->d.mat + md.mat0 + (long long)M_D * nn, nn * sizeof(double),
                                cudaMemcpyDeviceToHost, b->stream));
        CUDA_OK(cudaStreamSynchronize(b->stream));
    }
    return RKS_OK;
}

extern "C" int64_t rks_batch_dump(rks_batch *b, int32_t m, int32_t what, void *out, int64_t cap) {
    if (!b || m < 0 || m >= b->nmol || !out) return RKS_EINVAL;
    CUDA_OK(cudaStreamSynchronize(b->stream));
    const MolDesc &md = b->md[m];
    const DevBatch &d = b->d;
    const long long nn = (long long)md.nbf * md.nbf;
    MolState st;
    CUDA_OK(cudaMemcpy(&st, d.st + m, sizeof st, cudaMemcpyDeviceToHost));
    int npair = 0;
    CUDA_OK(cudaMemcpy(&npair, d.npair + m, sizeof(int), cudaMemcpyDeviceToHost));
    auto mat_dump = [&](int slot) -> int64_t {
        int64_t bytes = nn * sizeof(double);
        if (cap < bytes) return RKS_EINVAL;
        cudaError_t e = cudaMemcpy(out, d.mat + md.mat0 + (long long)slot * nn, bytes, cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? bytes : (int64_t)rks_cuda_fail(e, "dump", __FILE__, __LINE__);
    };
    switch (what) {
    case RKS_DUMP_PAIRS: {
        int64_t bytes = (int64_t)npair * 8;
        if (cap < bytes) return RKS_EINVAL;
        CUDA_OK(cudaMemcpy(out, d.kpair + md.pair0, bytes, cudaMemcpyDeviceToHost));
        return bytes;
    }
    case RKS_DUMP_PAIR_Q: {
        int64_t bytes = (int64_t)npair * 8;
        if (cap < bytes) return RKS_EINVAL;
        CUDA_OK(cudaMemcpy(out, d.kq + md.pair0, bytes, cudaMemcpyDeviceToHost));
        return bytes;
    }
    case RKS_DUMP_ROW_OFF: {
        int64_t bytes = (int64_t)(npair + 1) * 8;
        if (cap < bytes) return RKS_EINVAL;
        CUDA_OK(cudaMemcpy(out, d.row_off + md.pair0 + m, bytes, cudaMemcpyDeviceToHost));
        return bytes;
    }
    case RKS_DUMP_QUARTETS: {
        int64_t bytes = (int64_t)npair * 4;
        if (cap < bytes) return RKS_EINVAL;
        CUDA_OK(cudaMemcpy(out, d.row_nq + md.pair0, bytes, cudaMemcpyDeviceToHost));
        return bytes;
    }
    case RKS_DUMP_STORE: {
        if (b->direct) return fail(RKS_EINVAL, "direct SCF keeps no packed store");
        long long n = st.n_elem;
        int64_t bytes = n * 8;
        if (cap < bytes) return RKS_EINVAL;
        if (b->precision) {
            std::vector<float> tmp(n);
            CUDA_OK(cudaMemcpy(tmp.data(), (float *)d.store + md.eri0, n * 4, cudaMemcpyDeviceToHost));
            for (long long i = 0; i < n; i++) ((double *)out)[i] = tmp[i];
        } else {
            CUDA_OK(cudaMemcpy(out, (double *)d.store + md.eri0, bytes, cudaMemcpyDeviceToHost));
        }
        return bytes;
    }
    case RKS_DUMP_S: return mat_dump(M_S);
    case RKS_DUMP_T: return mat_dump(M_T);
    case RKS_DUMP_V: return mat_dump(M_V);
    case RKS_DUMP_J: return mat_dump(M_J);
    case RKS_DUMP_K: return mat_dump(M_K);
    case RKS_DUMP_VXC: return mat_dump(M_VXC);
    case RKS_DUMP_D: return mat_dump(M_D);
    case RKS_DUMP_F: return mat_dump(M_F);
    case RKS_DUMP_X: return mat_dump(M_X);
    case RKS_DUMP_EPS: {
        int64_t bytes = md.nbf * 8;
        if (cap < bytes) return RKS_EINVAL;
        memcpy(out, st.eps, bytes);
        return bytes;
    }
    case RKS_DUMP_GRID: {
        // stored as offsets from the owning nucleus; returned as absolute positions
        int64_t bytes = (int64_t)md.npts * 32;
        if (cap < bytes) return RKS_EINVAL;
        const size_t esz = b->precision ? 4 : 8;
        std::vector<unsigned char> t(md.npts * esz);
        std::vector<double> ax(3 * md.natom);
        CUDA_OK(cudaMemcpy(ax.data(), d.axyz + 3 * md.atom0, ax.size() * 8, cudaMemcpyDeviceToHost));
        const int npa = d.n_rad * d.n_theta * d.n_phi;
        void *src[4] = {d.gx, d.gy, d.gz, d.gw};
        for (int k = 0; k < 4; k++) {
            CUDA_OK(cudaMemcpy(t.data(), (unsigned char *)src[k] + md.pts0 * esz, md.npts * esz, cudaMemcpyDeviceToHost));
            for (int i = 0; i < md.npts; i++) {
                double v = esz == 4 ? (double)((float *)t.data())[i] : ((double *)t.data())[i];
                if (k < 3) v += ax[3 * (i / npa) + k];
                ((double *)out)[4 * i + k] = v;
            }
        }
        return bytes;
    }
    case RKS_DUMP_SCALARS: {
        if (cap < 80) return RKS_EINVAL;
        double *o = (double *)out;
        o[0] = st.E; o[1] = st.Exc; o[2] = st.Enuc; o[3] = md.npair_all; o[4] = st.n_quartets;
        o[5] = (double)st.n_elem; o[6] = md.npts; o[7] = st.near_ties;
        o[8] = st.grid_pairs[0]; o[9] = st.grid_pairs[1];
        return 80;
    }
    default: return RKS_EINVAL;
    }
}

// -------------------------------------------------------- unit entries
// Arguments of the unit entries, checked the same way by every variant.
static int check_unit_precision(int32_t precision) {
    if (precision != RKS_FP64 && precision != RKS_MIXED) return fail(RKS_EINVAL, "precision must be RKS_FP64 or RKS_MIXED");
    return RKS_OK;
}

extern "C" int rks_eval_boys(rks_ctx *ctx, int32_t mmax, int32_t n, const double *T, double *out, int32_t precision) {
    if (!ctx || n <= 0 || !T || !out || mmax < 0 || mmax > 4) return fail(RKS_EINVAL, "null argument, n <= 0 or mmax");
    int rc = check_unit_precision(precision);
    if (rc) return rc;
    double *dT = nullptr, *dO = nullptr;
    cudaStream_t st = ctx->stream;
    // every device step on the context stream: a legacy-stream copy from
    // pageable memory may return before its DMA lands, and that stream does
    // not order the kernel
    cudaError_t e = cudaMalloc(&dT, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dO, (size_t)n * (mmax + 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dT, T, n * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        launch_boys_eval(mmax, n, dT, dO, precision == RKS_MIXED, ctx->boys64, ctx->boys32, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, dO, (size_t)n * (mmax + 1) * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    else cudaStreamSynchronize(st);  // nothing queued may still use the buffers freed below
    cudaFree(dT);
    cudaFree(dO);
    return e == cudaSuccess ? RKS_OK : rks_cuda_fail(e, "rks_eval_boys", __FILE__, __LINE__);
}

extern "C" int rks_eval_xc(rks_ctx *ctx, int32_t n, const double *rho, const double *sigma, double *e, double *vr,
                           double *vs, int32_t precision) {
    if (!ctx || n <= 0 || !rho || !sigma || !e || !vr || !vs) return fail(RKS_EINVAL, "null argument or n <= 0");
    int rc = check_unit_precision(precision);
    if (rc) return rc;
    double *dr = nullptr, *ds = nullptr, *dO = nullptr;
    cudaStream_t st = ctx->stream;
    cudaError_t err = cudaMalloc(&dr, n * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc(&ds, n * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc(&dO, 3ull * n * sizeof(double));
    if (err == cudaSuccess) err = cudaMemcpyAsync(dr, rho, n * sizeof(double), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaMemcpyAsync(ds, sigma, n * sizeof(double), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) {
        launch_eval_xc(n, dr, ds, dO, precision == RKS_MIXED, st);
        err = cudaGetLastError();
    }
    double *outs[3] = {e, vr, vs};
    for (int k = 0; k < 3 && err == cudaSuccess; k++)
        err = cudaMemcpy2DAsync(outs[k], sizeof(double), dO + k, 3 * sizeof(double), sizeof(double), n,
                                cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    else cudaStreamSynchronize(st);  // drain before the buffers are freed
    cudaFree(dr);
    cudaFree(ds);
    cudaFree(dO);
    return err == cudaSuccess ? RKS_OK : rks_cuda_fail(err, "rks_eval_xc", __FILE__, __LINE__);
}

extern "C" int rks_probe_peak(rks_ctx *ctx, int32_t kind, double *ops_per_s) {
    if (!ctx || !ops_per_s || kind < RKS_PROBE_FP32_FMA || kind > RKS_PROBE_TF32_MMA)
        return fail(RKS_EINVAL, "null argument or unknown probe kind");
    CUDA_OK(cudaSetDevice(ctx->opt.device));
    int rc = probe_rate(kind, ctx->stream, ops_per_s);
    if (rc == RKS_EDEVICE) return fail(rc, "probe: bounded wait gave up");
    return rc;
}

extern "C" int rks_selftest_bounded_wait(rks_ctx *ctx, int32_t spins) {
    if (!ctx || spins <= 0 || spins > (1 << 24)) return fail(RKS_EINVAL, "spins out of range");
    int *d = nullptr, h = 0;
    CUDA_OK(cudaMalloc(&d, sizeof(int)));
    launch_wait_selftest(d, spins, ctx->stream);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    if (e != cudaSuccess) return rks_cuda_fail(e, "bounded-wait self test", __FILE__, __LINE__);
    return h ? fail(RKS_EDEVICE, "bounded wait gave up (expected: nothing arrives)") : RKS_OK;
}

// ------------------------------------------- allocation-free XC entry
// The same B3LYP kernel as rks_eval_xc, staged through one file-scope device
// array instead of cudaMalloc'd buffers.  For callers that must not allocate:
// a process whose device memory is already promised to the serving budget
// (a cudaMalloc could fail or push a cohort out), or one with cohorts in
// flight, where cudaFree would wait for the whole device.  Layout of the
// scratch: rho[MAX] | sigma[MAX] | out[3 * MAX] (e, v_rho, v_sigma
// interleaved per point).  Nothing in it needs to start at zero: every
// element a call reads was written earlier in that call.
static __device__ __align__(256) double g_xc_scratch[5 * RKS_XC_NOALLOC_MAX];

#define RKS_MAX_DEVICES 64
static std::mutex g_xc_scratch_mu[RKS_MAX_DEVICES];      // one scratch per device: its calls are serialised
static double *g_xc_scratch_ptr[RKS_MAX_DEVICES] = {};   // device address per ordinal, looked up on first use

extern "C" int rks_eval_xc_noalloc(rks_ctx *ctx, int32_t n, const double *rho, const double *sigma, double *e,
                                   double *vr, double *vs, int32_t precision) {
    if (!ctx || n <= 0 || !rho || !sigma || !e || !vr || !vs) return fail(RKS_EINVAL, "null argument or n <= 0");
    if (n > RKS_XC_NOALLOC_MAX)
        return fail(RKS_EINVAL, "n = " + std::to_string(n) + " exceeds the static scratch (RKS_XC_NOALLOC_MAX = " +
                                    std::to_string(RKS_XC_NOALLOC_MAX) + " points)");
    int rc = check_unit_precision(precision);
    if (rc) return rc;
    const int dev = ctx->opt.device;
    if (dev < 0 || dev >= RKS_MAX_DEVICES) return fail(RKS_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_xc_scratch_mu[dev]);
    int prev = 0;
    CUDA_OK(cudaGetDevice(&prev));
    if (prev != dev) CUDA_OK(cudaSetDevice(dev));
    double *base = g_xc_scratch_ptr[dev];
    cudaError_t err = cudaSuccess;
    if (!base) {
        // set-up, once per device, with that device current
        err = cudaGetSymbolAddress((void **)&base, g_xc_scratch);
        if (err == cudaSuccess) g_xc_scratch_ptr[dev] = base;
    }
    if (err == cudaSuccess) {
        double *dr = base, *ds = base + RKS_XC_NOALLOC_MAX, *dO = base + 2 * RKS_XC_NOALLOC_MAX;
        cudaStream_t st = ctx->stream;
        err = cudaMemcpyAsync(dr, rho, n * sizeof(double), cudaMemcpyHostToDevice, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(ds, sigma, n * sizeof(double), cudaMemcpyHostToDevice, st);
        if (err == cudaSuccess) {
            launch_eval_xc(n, dr, ds, dO, precision == RKS_MIXED, st);
            err = cudaGetLastError();
        }
        double *outs[3] = {e, vr, vs};
        for (int k = 0; k < 3 && err == cudaSuccess; k++)
            err = cudaMemcpy2DAsync(outs[k], sizeof(double), dO + k, 3 * sizeof(double), sizeof(double), n,
                                    cudaMemcpyDeviceToHost, st);
        // on an error after the first enqueue, drain the stream anyway: the
        // lock is released on return, and the next holder must find the
        // scratch idle
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        else cudaStreamSynchronize(st);
    }
    if (err != cudaSuccess) rc = rks_cuda_fail(err, "rks_eval_xc_noalloc", __FILE__, __LINE__);
    if (prev != dev) cudaSetDevice(prev);
    return rc;
}

// ----------------------------------------------------- serving worker
// Continuous batching.  The worker keeps up to max_cohorts batches in flight,
// each on its own stream, so a request that arrives while others are
// mid-SCF starts at once instead of waiting for the running batch to finish.
// Each pass of the loop (1) admits queued molecules as a new cohort when the
// HBM budget has room, (2) advances every cohort whose last enqueued chunk has
// completed (CUDA event query, no blocking): a few more SCF iterations, or the
// final step once its pinned active count reads zero (or the protocol's
// iteration count is reached), and (3) retires cohorts whose final step is
// done: results go to their tickets and the memory returns to the budget.
struct Cohort {
    rks_batch *b = nullptr;
    std::vector<uint64_t> ids;
    int phase = 0;  // 0 iterating, 2 recheck marked, 3 rechecking, 1 final step enqueued
    int rc_enq = 0; // recheck iterations enqueued
    int n_precise = 0;
    bool counted = false;  // the last chunk ended with an active-count readback
    cudaEvent_t ev = nullptr;
};

static void fail_tickets(rks_ctx *c, const std::vector<uint64_t> &ids, int err = RKS_ECUDA) {
    std::lock_guard<std::mutex> lk(c->mu);
    for (auto id : ids) {
        auto it = c->tickets.find(id);
        if (it != c->tickets.end()) {
            it->second.state = RKS_FAILED;
            it->second.err = err;
        }
    }
    c->cv_done.notify_all();
}

// Enqueue the cohort's next chunk and record its event.
static int cohort_next(Cohort &h) {
    rks_batch *b = h.b;
    const DevBatch &d = b->d;
    int rc = RKS_OK;
    if (h.phase == 2) {
        // the marked counts have landed in the pinned words (the chunk's event completed)
        const int n_precise = pinw(b)[0], n_fp64 = pinw(b)[1];
        if (n_fp64 > 0) rc = start_fp64_redo(b, n_fp64);
        if (!rc && n_precise > 0) {
            h.phase = 3;
            h.n_precise = n_precise;
            const int k = std::min(kCheckEvery, d.fixed_iters);
            b->n_precise = n_precise;
            rc = enqueue_iters(b, k, kPrecise);
            b->n_precise = 0;
            h.rc_enq = k;
        } else if (!rc) {
            rc = enqueue_final(b);
            if (!rc) rc = enqueue_adopt(b);
            h.phase = 1;
        }
    } else if (h.phase == 3) {
        if (h.rc_enq >= d.fixed_iters) {
            rc = enqueue_final(b);
            if (!rc) rc = enqueue_adopt(b);
            h.phase = 1;
        } else {
            const int k = std::min(kCheckEvery, d.fixed_iters - h.rc_enq);
            b->n_precise = h.n_precise;
            rc = enqueue_iters(b, k, kPrecise);
            b->n_precise = 0;
            h.rc_enq += k;
        }
    } else if (h.phase == 0) {
        bool done;
        if (d.fixed_iters > 0) done = b->it_enq >= d.fixed_iters;
        else done = b->it_enq >= d.max_iters || (h.counted && pinw(b)[0] == 0);
        if (done && recheck_on(b)) {
            rc = enqueue_recheck_start(b);
            h.phase = 2;
        } else if (done) {
            rc = enqueue_final(b);
            if (!rc) rc = enqueue_adopt(b);
            h.phase = 1;
        } else {
            const int lim = d.fixed_iters > 0 ? d.fixed_iters : d.max_iters;
            rc = enqueue_iters(b, std::min(kCheckEvery, lim - b->it_enq), iter_prec(b));
            if (!rc && d.fixed_iters == 0) {
                rc = enqueue_active_count(b);
                h.counted = true;
            }
        }
    }
    if (rc) return rc;
    CUDA_OK(cudaEventRecord(h.ev, b->stream));
    return RKS_OK;
}

static int cohort_start(rks_ctx *c, Cohort &h, const std::vector<int32_t> &na, const std::vector<int32_t> &Z,
                        const std::vector<double> &xyz) {
    cudaStream_t st = nullptr;
    CUDA_OK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    int rc = batch_create_on(c, st, true, (int)na.size(), na.data(), Z.data(), xyz.data(), &h.b);
    if (rc) return rc;
    if ((rc = rks_batch_setup(h.b))) return rc;
    CUDA_OK(cudaEventCreateWithFlags(&h.ev, cudaEventDisableTiming));
    return cohort_next(h);
}

static void cohort_free(Cohort &h) {
    if (h.b) rks_batch_destroy(h.b);
    if (h.ev) cudaEventDestroy(h.ev);
    h.b = nullptr;
    h.ev = nullptr;
}

// Copy results to the cohort's tickets (its stream is idle).
static void cohort_publish(rks_ctx *c, Cohort &h) {
    rks_batch *b = h.b;
    const int rc = rks_batch_sync(b);
    if (rc && rc != RKS_EDEVICE) {
        fail_tickets(c, h.ids);
        return;
    }
    std::vector<rks_result_t> res(h.ids.size());
    std::vector<std::vector<double>> eps(h.ids.size()), D(h.ids.size());
    std::vector<int> ok(h.ids.size(), 0);
    for (size_t k = 0; k < h.ids.size(); k++) {
        const int nbf = b->md[k].nbf;
        eps[k].resize(nbf);
        D[k].resize((size_t)nbf * nbf);
        ok[k] = rks_batch_result(b, (int)k, &res[k], eps[k].data(), D[k].data(), nbf) == RKS_OK;
    }
    std::lock_guard<std::mutex> lk(c->mu);
    auto now = std::chrono::steady_clock::now();
    for (size_t k = 0; k < h.ids.size(); k++) {
        auto it = c->tickets.find(h.ids[k]);
        if (it == c->tickets.end()) continue;
        Ticket &t = it->second;
        if (!ok[k]) {
            t.state = RKS_FAILED;
            continue;
        }
        t.res = res[k];
        t.res.latency_s = std::chrono::duration<double>(now - t.t_submit).count();
        t.eps.swap(eps[k]);
        t.D.swap(D[k]);
        t.state = RKS_DONE;
    }
    c->cv_done.notify_all();
}

static void worker_main(rks_ctx *c) {
    cudaSetDevice(c->opt.device);
    std::vector<Cohort> live;
    const auto admit_wait = std::chrono::microseconds(std::max(0, c->opt.admit_wait_us));
    for (;;) {
        // (1) admission
        std::vector<uint64_t> ids, rejected;
        std::vector<int32_t> na, Z;
        std::vector<double> xyz;
        {
            std::unique_lock<std::mutex> lk(c->mu);
            if (live.empty()) c->cv.wait(lk, [&] { return c->stop || !c->queue.empty(); });
            if (c->stop) break;
            size_t inflight = 0;
            for (auto &h : live) inflight += h.b->bytes;
            const bool room = (int)live.size() < std::max(1, c->opt.max_cohorts);
            bool admit = room && !c->queue.empty();
            if (admit && !live.empty() && (int)c->queue.size() < c->opt.max_slots) {
                auto waited = std::chrono::steady_clock::now() - c->tickets[c->queue.front()].t_submit;
                admit = waited >= admit_wait;
            }
            size_t need = 0;
            while (admit && !c->queue.empty() && (int)ids.size() < c->opt.max_slots) {
                const uint64_t id = c->queue.front();
                Ticket &t = c->tickets[id];
                const size_t mb = mol_bytes(c->opt, (int)t.Z.size(), t.Z.data());
                if (inflight + need + mb > c->budget) {
                    // larger than the whole budget: it can never run
                    if (live.empty() && ids.empty()) {
                        c->queue.pop_front();
                        rejected.push_back(id);
                        continue;
                    }
                    break;
                }
                need += mb;
                c->queue.pop_front();
                ids.push_back(id);
                t.state = RKS_RUNNING;
                na.push_back((int)t.Z.size());
                Z.insert(Z.end(), t.Z.begin(), t.Z.end());
                xyz.insert(xyz.end(), t.xyz.begin(), t.xyz.end());
            }
        }
        if (!rejected.empty()) fail_tickets(c, rejected, RKS_ENOMEM);
        bool progressed = !ids.empty();
        if (!ids.empty()) {
            Cohort h;
            h.ids = ids;
            if (cohort_start(c, h, na, Z, xyz) == RKS_OK) {
                live.push_back(h);
            } else {
                fail_tickets(c, h.ids);
                cohort_free(h);
            }
        }
        // (2) advance, (3) retire
        for (size_t k = 0; k < live.size();) {
            Cohort &h = live[k];
            const cudaError_t q = cudaEventQuery(h.ev);
            if (q == cudaErrorNotReady) {
                k++;
                continue;
            }
            progressed = true;
            int rc = q == cudaSuccess ? RKS_OK : rks_cuda_fail(q, "cohort", __FILE__, __LINE__);
            if (!rc && h.phase != 1) rc = cohort_next(h);
            else if (!rc) {
                cohort_publish(c, h);
                cohort_free(h);
                live.erase(live.begin() + k);
                continue;
            }
            if (rc) {
                fail_tickets(c, h.ids);
                cohort_free(h);
                live.erase(live.begin() + k);
                continue;
            }
            k++;
        }
        if (!progressed) {
            std::unique_lock<std::mutex> lk(c->mu);
            if (!c->stop) c->cv.wait_for(lk, std::chrono::microseconds(200));
        }
    }
    for (auto &h : live) {
        fail_tickets(c, h.ids);
        cohort_free(h);
    }
}

extern "C" int rks_create(const rks_options *options, rks_ctx **out) {
    if (!out) return RKS_EINVAL;
    std::call_once(g_basis_once, init_basis);
    rks_options o;
    if (options) o = *options; else rks_options_default(&o);
    if (o.basis != 0 || o.n_rad <= 0 || o.n_theta <= 0 || o.n_theta > 64 || o.n_phi <= 0 || o.becke_iters < 0 ||
        (o.precision != RKS_FP64 && o.precision != RKS_MIXED) || o.max_iters <= 0 || o.max_slots <= 0 ||
        !(o.fix_theta >= 0) || (o.guess != RKS_GUESS_SAD && o.guess != RKS_GUESS_CORE) || o.max_cohorts <= 0 ||
        o.iter_precision < 0 || o.iter_precision > 3 || !(o.recheck_err >= 0) || !(o.recheck_fp64_err >= 0) ||
        o.admit_wait_us < 0 || o.grid_chunks < 0 || o.grid_chunks > 256 || o.jk_chunks < 0 || o.jk_chunks > 256 ||
        o.direct_scf < RKS_DIRECT_NEVER || o.direct_scf > RKS_DIRECT_AUTO)
        return fail(RKS_EINVAL, "bad options");
    int ndev = 0;
    CUDA_OK(cudaGetDeviceCount(&ndev));
    if (o.device < 0 || o.device >= ndev) return fail(RKS_EINVAL, "no such device");
    CUDA_OK(cudaSetDevice(o.device));
    rks_ctx *c = new rks_ctx();
    c->opt = o;
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, o.device);
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&c->boys64, sizeof(double) * BOYS_N64 * BOYS_COL64);
    if (e == cudaSuccess) e = cudaMalloc(&c->boys32, sizeof(float) * BOYS_N32 * BOYS_COL32);
    if (e == cudaSuccess) e = cudaMalloc(&c->rad, sizeof(double) * 5 * o.n_rad * 2);
    if (e == cudaSuccess) e = cudaMalloc(&c->ang, sizeof(double) * o.n_theta * o.n_phi * 4);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&c->pin, sizeof(int) * 2 * kPinSlots, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        delete c;
        return rks_cuda_fail(e, "context allocation", __FILE__, __LINE__);
    }
    launch_boys_table(c->boys64, c->boys32, c->stream);
    launch_quad_tables(c->rad, c->ang, o.n_rad, o.n_theta, o.n_phi, c->stream);
    e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        delete c;
        return rks_cuda_fail(e, "context tables", __FILE__, __LINE__);
    }
    for (int k = kPinSlots - 1; k >= 0; k--) c->pin_free.push_back(k);
    if (o.hbm_budget_bytes) {
        c->budget = o.hbm_budget_bytes;
    } else {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        c->budget = (size_t)(0.85 * (double)fr);
    }
    c->worker = std::thread(worker_main, c);
    *out = c;
    return RKS_OK;
}

extern "C" int rks_destroy(rks_ctx *c) {
    if (!c) return RKS_EINVAL;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->stop = true;
        for (auto id : c->queue) c->tickets[id].state = RKS_FAILED;
        c->queue.clear();
    }
    c->cv.notify_all();
    if (c->worker.joinable()) c->worker.join();
    cudaStreamSynchronize(c->stream);
    for (auto &r : c->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    cudaFree(c->boys64);
    cudaFree(c->boys32);
    cudaFree(c->rad);
    cudaFree(c->ang);
    if (c->pin) cudaFreeHost(c->pin);
    cudaStreamDestroy(c->stream);
    delete c;
    return RKS_OK;
}

extern "C" int rks_submit(rks_ctx *c, int32_t natom, const int32_t *Z, const double *xyz, uint64_t *ticket_out) {
    if (!c || !ticket_out) return RKS_EINVAL;
    int rc = validate(natom, Z, xyz, nullptr);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->queue.size() >= c->queue_cap) return RKS_EAGAIN;
    uint64_t id = c->next_ticket++;
    Ticket &t = c->tickets[id];
    t.Z.assign(Z, Z + natom);
    t.xyz.assign(xyz, xyz + 3 * natom);
    t.t_submit = std::chrono::steady_clock::now();
    c->queue.push_back(id);
    *ticket_out = id;
    c->cv.notify_one();
    return RKS_OK;
}

extern "C" int rks_submit_batch(rks_ctx *c, int32_t nmol, const int32_t *natom, const int32_t *Z,
                                const double *xyz, uint64_t *tickets_out) {
    if (!c || nmol < 0 || (nmol > 0 && (!natom || !Z || !xyz || !tickets_out))) return RKS_EINVAL;
    long long off = 0;
    for (int m = 0; m < nmol; m++) {
        int rc = validate(natom[m], Z + off, xyz + 3 * off, nullptr);
        if (rc) return fail(rc, "molecule " + std::to_string(m) + ": " + g_err);
        off += natom[m];
    }
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->queue.size() + (size_t)nmol > c->queue_cap) return RKS_EAGAIN;
    const auto now = std::chrono::steady_clock::now();
    off = 0;
    for (int m = 0; m < nmol; m++) {
        const uint64_t id = c->next_ticket++;
        Ticket &t = c->tickets[id];
        t.Z.assign(Z + off, Z + off + natom[m]);
        t.xyz.assign(xyz + 3 * off, xyz + 3 * (off + natom[m]));
        t.t_submit = now;
        c->queue.push_back(id);
        tickets_out[m] = id;
        off += natom[m];
    }
    c->cv.notify_one();
    return RKS_OK;
}

extern "C" int rks_poll(rks_ctx *c, uint64_t ticket, int32_t *state_out) {
    if (!c || !state_out) return RKS_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->tickets.find(ticket);
    if (it == c->tickets.end()) return RKS_ENOTFOUND;
    *state_out = it->second.state;
    return RKS_OK;
}

extern "C" int rks_wait(rks_ctx *c, uint64_t ticket, double timeout_s) {
    if (!c) return RKS_EINVAL;
    std::unique_lock<std::mutex> lk(c->mu);
    auto done = [&] {
        auto it = c->tickets.find(ticket);
        return it == c->tickets.end() || it->second.state == RKS_DONE || it->second.state == RKS_FAILED;
    };
    if (!c->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) return RKS_ETIMEOUT;
    if (c->tickets.find(ticket) == c->tickets.end()) return RKS_ENOTFOUND;
    return RKS_OK;
}

extern "C" int rks_result(rks_ctx *c, uint64_t ticket, rks_result_t *out, double *eps_out, double *D_out,
                          int32_t cap_nbf) {
    if (!c || !out) return RKS_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->tickets.find(ticket);
    if (it == c->tickets.end()) return RKS_ENOTFOUND;
    Ticket &t = it->second;
    if (t.state == RKS_FAILED) {
        const int err = t.err;
        c->tickets.erase(it);
        return fail(err, err == RKS_ENOMEM ? "molecule exceeds the HBM budget" : "ticket failed");
    }
    if (t.state != RKS_DONE) return RKS_ENOTREADY;
    if ((eps_out || D_out) && cap_nbf < t.res.nbf) return RKS_EINVAL;
    *out = t.res;
    if (eps_out) memcpy(eps_out, t.eps.data(), sizeof(double) * t.eps.size());
    if (D_out) memcpy(D_out, t.D.data(), sizeof(double) * t.D.size());
    c->tickets.erase(it);
    return RKS_OK;
}
