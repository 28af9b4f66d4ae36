// C ABI and host runtime of the GB300 l-marginal L1 Sinkhorn library
// (arXiv 2405.19246).  See include/mmot.h for the contract of every call.
//
// Plan layout in device memory (one plan = one problem instance):
//   merged order of all T = sum_k N_k points (Eq. D_p tie rule), struct of arrays
//     pos   FP32 [T]  (x_t - x_first_of_tile)/eps   (FP64 in the all-FP64 path)
//     mid   u8   [T]  marginal of the point
//     lphi  FP32 [T]  g_m(i)/eps - beta[tile][m]  (re-centred ln phi, Algorithm 5 idea;
//                     FP64 in the all-FP64 path)
//   per tile: first index, first/last x (FP64), span, per-marginal counts before
//     the tile, reference tile for each marginal's baseline, baselines beta (FP64)
//   per marginal: g_k (FP64 potentials), mu_k and ln mu_k (FP64)
//   scan scratch: per-tile aggregates / inclusive prefixes / flags, backward
//     carries, residual partial sums.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/mmot.h"
#include "mmot_internal.cuh"
#include "layout.h"
#include "shapes.cuh"

using namespace mmot;

namespace {

thread_local std::string g_last_error;

// process-wide cap on the device bytes held by plans (0: none) and the bytes
// they hold now
std::atomic<int64_t> g_mem_limit{0};
std::atomic<int64_t> g_mem_used{0};

}  // namespace

namespace mmot {
mmot_status set_error(mmot_status st, const char *msg)
{
    g_last_error = msg;
    return st;
}
}  // namespace mmot

namespace {

mmot_status fail(mmot_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define CUDA_TRY(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            cudaGetLastError(); /* do not leave a non-sticky error for the next check */      \
            return fail(e_ == cudaErrorMemoryAllocation ? MMOT_ERR_OOM : MMOT_ERR_CUDA,       \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                                     \
    } while (0)

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Kahan-compensated sum of per-tile partial sums (one block).
__global__ void k_sum_partials(const double *partial, int n, double *out, int accumulate)
{
    __shared__ double s_sum[256];
    __shared__ double s_c[256];
    double sum = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double y = partial[i] - c;
        const double t = sum + y;
        c = (t - sum) - y;
        sum = t;
    }
    s_sum[threadIdx.x] = sum;
    s_c[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0, Cc = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const double y = s_sum[i] - s_c[i] - Cc;
            const double t = S + y;
            Cc = (t - S) - y;
            S = t;
        }
        out[0] = accumulate ? out[0] + S : S;
    }
}

}  // namespace

// One problem instance as given to plan creation (host or device pointers).
struct InstanceIn {
    const int64_t *N = nullptr;
    const double *const *x = nullptr;
    const double *const *mu = nullptr;
    double eps = 0.0;
    // shards of one instance: the sizes of the whole instance (initial
    // potentials -eps ln N_total); the shard's weights need not sum to 1
    const int64_t *Ntot = nullptr;
    double init_count(int k) const { return (double)(Ntot ? Ntot[k] : N[k]); }
};

struct mmot_plan_s {
    int l = 0;
    int64_t N[MMOT_MAXL] = {0};
    int64_t T = 0;
    double eps = 0;
    int prec = 1;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int nt = 0;
    int NB = 0;
    int NS = 0;
    int K = 0;
    int NT = 0;
    int check_every = 10;
    int spin_limit = 1 << 23;
    int use_graph = 1;
    int hold = 0;           // test hook (MMOT_OPT_TEST_HOLD)
    // shard of one instance (mmot_shard_create): states entering the range
    // for target inflow_target ([2][NS] scaled floats), composed operator out
    bool shard = false;
    int64_t Ninit[MMOT_MAXL] = {0};
    unsigned char *inflow = nullptr;
    int inflow_target = -1;
    double *d_lnop = nullptr;   // [2][NB+1][NS]
    int64_t dev_bytes = 0;  // device memory held by this plan
    // host copies needed to re-centre potentials
    HVec<uint8_t> h_mid;
    HVec<uint32_t> h_tile_of;          // tile of each merged point
    HVec<uint32_t> h_mpos[MMOT_MAXL];  // merged index of each local point
    std::vector<uint32_t> h_tstart;
    std::vector<uint32_t> h_toff;   // padded stream offset of each tile (l <= 5)
    std::vector<int32_t> h_reftile;
    std::vector<double> h_beta;
    std::vector<double> h_beta0;   // baselines of the initial potentials
    // batches: instances laid out one after the other (nseg = 1: single problem)
    int nseg = 1;
    bool batch = false;               // created by mmot_batch_create
    std::vector<int32_t> seg_tile0;   // [nseg+1] first tile of each instance
    std::vector<int64_t> seg_off;     // [(nseg+1)*l] first local index of instance q in marginal k
    std::vector<double> seg_eps;      // [nseg]
    std::vector<int64_t> seg_N;       // [nseg*l]
    int32_t *d_seg = nullptr;         // [nt] instance of each tile
    double *d_teps = nullptr;         // [nt] eps of each tile
    int32_t *d_frozen = nullptr;      // [nseg] converged instances (no more updates)
    int32_t *d_segt0 = nullptr;       // [nseg+1]
    double *d_res = nullptr;          // [nseg] per-instance residuals
    int64_t *d_goff = nullptr;        // [(nseg+1)*l] copy of seg_off
    double *d_g0 = nullptr;           // [nseg*l] initial potential value per instance and marginal
    // device
    void *pos = nullptr;     // FP32 or FP64 (esz bytes per point)
    uint8_t *mid = nullptr;
    void *lphi = nullptr;    // FP32 or FP64
    size_t esz = 4;
    uint32_t *tstart = nullptr;
    double *ulb = nullptr, *urb = nullptr;   // tile ends in units of eps
    double *span = nullptr;
    int32_t *cnt = nullptr, *reftile = nullptr;
    double *beta = nullptr;
    double *g[MMOT_MAXL] = {nullptr};
    double *lnmu[MMOT_MAXL] = {nullptr};
    float2 *lnmu_ff[MMOT_MAXL] = {nullptr};   // ln mu as FP32 hi + lo (FP32 path, l <= 5)
    // padded stream of the tile kernels (l <= 5): e^{pos}, scaled phi, marginal
    int64_t Tpad = 0;
    uint32_t *toff = nullptr;
    void *epos = nullptr, *ephi = nullptr;
    uint8_t *emid = nullptr;
    double *mu[MMOT_MAXL] = {nullptr};
    // scaled floats: float2 (FP32 path) or double2 (FP64 path), sfsz bytes each
    unsigned char *agg = nullptr, *inc = nullptr, *bcarry = nullptr;
    unsigned char *fcarry = nullptr, *opF = nullptr, *opB = nullptr;
    unsigned char *pdecF = nullptr, *pdecB = nullptr;
    unsigned char *coef = nullptr;   // level passes (l >= 6): per tile and marginal, level-to-level coefficients
    void *lops = nullptr;            // tile kernels (l <= 5): lanes' chunk operators of the current target
    void *ugrid = nullptr;           // uniform grid: e^{d h / eps} by grid steps d (no epos / emid)
    void *gtarg = nullptr;           // warp tiles (l >= 6): backward states at the target points
    int *cflags = nullptr;          // carry-scan chunk flags
    size_t cflags_n = 0;
    unsigned char *cagg = nullptr;  // carry-scan chunk contributions [2][32][NS]
    size_t sfsz = 8;
    bool three_phase = false;  // tile operators + carry scan (l <= 5)
    int ops_target = -1;       // target whose tile operators are current
    double *partial = nullptr;
    double *part4 = nullptr;   // [nt*4] per-tile objective sums
    double *d_obj = nullptr;   // [nseg*6] per instance: mass, residual (all l), primal, g mu, W,
                               // residual of the stopping test (marginals 1..l-1)
    int *flags = nullptr;   // flags followed by the tile counter
    size_t flags_bytes = 0;
    int *err = nullptr;
    double *dsum = nullptr;  // reduction results
    double *scratch = nullptr;  // max N doubles
    cudaGraphExec_t graph = nullptr;
    // objective sweeps (l state bits, no target), device scratch allocated on
    // first use: tile operators, carries, decays and scan words
    bool obj_ready = false;
    std::vector<unsigned char> h_odecF, h_odecB;
    unsigned char *o_opF = nullptr, *o_opB = nullptr, *o_fc = nullptr, *o_bc = nullptr;
    unsigned char *o_decF = nullptr, *o_decB = nullptr, *o_cagg = nullptr, *o_agg = nullptr, *o_inc = nullptr;
    unsigned char *o_coef = nullptr;   // l = 8: per tile and marginal, the pair coefficient of a two-level pass
    int *o_cflags = nullptr, *o_flags = nullptr;
    size_t o_flags_bytes = 0;
    double *o_lnz = nullptr;   // [nt] ln Z seen by each tile
    std::vector<void *> allocs;
    // profiling: pairs of events around each kernel launch
    int profile = 0;
    struct Rec { int kernel; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    int64_t prof_count[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t launches = 0;   // kernels launched so far (graph replays included)
    double prof_ms[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};

    ~mmot_plan_s()
    {
        for (auto &r : recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        if (graph) cudaGraphExecDestroy(graph);
        for (void *p : allocs) cudaFree(p);
        g_mem_used -= dev_bytes;
        if (own_stream && st) cudaStreamDestroy(st);
    }

    template <typename Tp>
    cudaError_t alloc(Tp **p, size_t n)
    {
        void *q = nullptr;
        const int64_t bytes = (int64_t)(std::max<size_t>(1, n) * sizeof(Tp));
        const int64_t lim = g_mem_limit.load();
        if (lim > 0 && g_mem_used.load() + bytes > lim) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMalloc(&q, (size_t)bytes);
        if (e == cudaSuccess) {
            allocs.push_back(q);
            *p = static_cast<Tp *>(q);
            dev_bytes += bytes;
            g_mem_used += bytes;
        }
        return e;
    }
};

namespace {

// kind: 2 tile operators, 3 carry scan, 4 product
template <int NB>
cudaError_t launch_ops_nb(const SweepArgs &a, bool fp64, cudaStream_t st, int kind)
{
    if constexpr (NB <= kMaxOpBits) {
        if (fp64) {
            if (kind == 2) return launch_tileop<NB, double>(a, st);
            if (kind == 3) return launch_carry<NB, double>(a, st);
            return launch_prod<NB, double>(a, st);
        }
        if (kind == 2) return launch_tileop<NB, float>(a, st);
        if (kind == 3) return launch_carry<NB, float>(a, st);
        return launch_prod<NB, float>(a, st);
    } else {
        return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t mmot::launch_three_phase(int NB, const SweepArgs &a, bool fp64, cudaStream_t st, int kind)
{
    switch (NB) {
    case 1: return launch_ops_nb<1>(a, fp64, st, kind);
    case 2: return launch_ops_nb<2>(a, fp64, st, kind);
    case 3: return launch_ops_nb<3>(a, fp64, st, kind);
    case 4: return launch_ops_nb<4>(a, fp64, st, kind);
    default: return cudaErrorInvalidValue;
    }
}

namespace {

// kind 4: tile products (all NB); 5: level contributions, 6: level scan (NB >= 5)
template <int NB>
cudaError_t launch_lvl_nb(const SweepArgs &a, bool fp64, cudaStream_t st, int kind, int SL, int fwd)
{
    if constexpr (NB > kMaxOpBits) {
        if (kind == 4) return fp64 ? launch_prod<NB, double>(a, st) : launch_prod<NB, float>(a, st);
        if (kind == 5) return fp64 ? launch_lagg<NB, double>(a, st, SL, fwd) : launch_lagg<NB, float>(a, st, SL, fwd);
        if (kind == 6) return fp64 ? launch_lscan<NB, double>(a, st, SL, fwd) : launch_lscan<NB, float>(a, st, SL, fwd);
        if (kind == 7) return fp64 ? launch_wbwd<NB, double>(a, st) : launch_wbwd<NB, float>(a, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_levels(int NB, const SweepArgs &a, bool fp64, cudaStream_t st, int kind, int SL, int fwd)
{
    switch (NB) {
    case 5: return launch_lvl_nb<5>(a, fp64, st, kind, SL, fwd);
    case 6: return launch_lvl_nb<6>(a, fp64, st, kind, SL, fwd);
    case 7: return launch_lvl_nb<7>(a, fp64, st, kind, SL, fwd);
    default: return cudaErrorInvalidValue;
    }
}

template <int NB>
cudaError_t launch_opc_nb(const SweepArgs &a, bool fp64, cudaStream_t st, double *lnop)
{
    if constexpr (NB <= kMaxOpBits)
        return fp64 ? launch_opcompose<NB, double>(a, st, lnop) : launch_opcompose<NB, float>(a, st, lnop);
    return cudaErrorInvalidValue;
}

cudaError_t launch_opc(int NB, const SweepArgs &a, bool fp64, cudaStream_t st, double *lnop)
{
    switch (NB) {
    case 1: return launch_opc_nb<1>(a, fp64, st, lnop);
    case 2: return launch_opc_nb<2>(a, fp64, st, lnop);
    case 3: return launch_opc_nb<3>(a, fp64, st, lnop);
    case 4: return launch_opc_nb<4>(a, fp64, st, lnop);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ops(int NB, const SweepArgs &a, bool fp64, cudaStream_t st, int kind)
{
    return mmot::launch_three_phase(NB, a, fp64, st, kind);
}

template <typename V>
int wshape_k(int NB)
{
    switch (NB) {
    case 5: return WShape<5, V>::K;
    case 6: return WShape<6, V>::K;
    default: return WShape<7, V>::K;
    }
}

template <int NB>
void shape_nb(bool fp64, int *K, int *NT, int *JCAP)
{
    if (fp64) {
        *K = Shape<NB, double>::K;
        *NT = Shape<NB, double>::NT;
        *JCAP = Shape<NB, double>::JCAP;
    } else {
        *K = Shape<NB, float>::K;
        *NT = Shape<NB, float>::NT;
        *JCAP = Shape<NB, float>::JCAP;
    }
}

// lanes' chunk operators of one tile (tile.cuh): [dir][entry][lane]
int64_t tile_lops_bytes(int NB, bool fp64)
{
    int nop = 0;
    for (int s = 0; s < NB; ++s)
        for (int U = 1; U < (1 << NB); ++U)
            if (s + __builtin_popcount(U) <= NB) ++nop;
    int nt = 0;
    switch (NB) {
    case 1: nt = fp64 ? TShape<1, double>::NT : TShape<1, float>::NT; break;
    case 2: nt = fp64 ? TShape<2, double>::NT : TShape<2, float>::NT; break;
    case 3: nt = fp64 ? TShape<3, double>::NT : TShape<3, float>::NT; break;
    default: nt = fp64 ? TShape<4, double>::NT : TShape<4, float>::NT; break;
    }
    return (int64_t)2 * nop * nt * (fp64 ? 8 : 4);
}

int tile_jcap(int NB, bool fp64)
{
    switch (NB) {
    case 1: return fp64 ? TShape<1, double>::JCAP : TShape<1, float>::JCAP;
    case 2: return fp64 ? TShape<2, double>::JCAP : TShape<2, float>::JCAP;
    case 3: return fp64 ? TShape<3, double>::JCAP : TShape<3, float>::JCAP;
    default: return fp64 ? TShape<4, double>::JCAP : TShape<4, float>::JCAP;
    }
}

void shape_of(int NB, bool fp64, int *K, int *NT, int *JCAP)
{
    switch (NB) {
    case 1: shape_nb<1>(fp64, K, NT, JCAP); break;
    case 2: shape_nb<2>(fp64, K, NT, JCAP); break;
    case 3: shape_nb<3>(fp64, K, NT, JCAP); break;
    case 4: shape_nb<4>(fp64, K, NT, JCAP); break;
    case 5: shape_nb<5>(fp64, K, NT, JCAP); break;
    case 6: shape_nb<6>(fp64, K, NT, JCAP); break;
    default: shape_nb<7>(fp64, K, NT, JCAP); break;
    }
}

SweepArgs make_args(mmot_plan p, int j, int mode, double *out)
{
    SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.l = p->l;
    a.j = j;
    a.nt = p->nt;
    a.mode = mode;
    a.spin_limit = p->spin_limit;
    a.hold = p->hold;
    a.eps = p->eps;
    a.inv_eps = 1.0 / p->eps;
    a.tstart = p->tstart;
    a.ulb = p->ulb;
    a.urb = p->urb;
    a.span = p->span;
    a.cnt = p->cnt;
    a.reftile = p->reftile;
    a.beta = p->beta;
    a.pos = p->pos;
    a.mid = p->mid;
    a.lphi = p->lphi;
    a.agg = p->agg;
    a.inc = p->inc;
    a.flags = p->flags;
    a.counter = p->flags + (size_t)p->nt * (p->NB + 1);
    a.bcarry = p->bcarry;
    a.fcarry = p->fcarry;
    a.opF = p->opF;
    a.opB = p->opB;
    a.pdecF = p->pdecF;
    a.pdecB = p->pdecB;
    a.cflags = p->cflags;
    a.cagg = p->cagg;
    a.toff = p->toff;
    a.epos = p->epos;
    a.ephi = p->ephi;
    a.emid = p->emid;
    a.lnmuj_ff = (j < p->l) ? p->lnmu_ff[j] : nullptr;
    a.jnext = -1;
    // j = l: no target marginal (objective sweeps)
    a.gj = (j < p->l) ? p->g[j] : nullptr;
    a.lnmuj = (j < p->l) ? p->lnmu[j] : nullptr;
    a.muj = (j < p->l) ? p->mu[j] : nullptr;
    a.out = out;
    a.partial = p->partial;
    a.part4 = p->part4;
    a.err = p->err;
    a.seg = p->d_seg;
    a.teps = p->d_teps;
    a.frozen = p->d_frozen;
    a.inflow = (p->shard && j < p->l && p->inflow_target == j) ? p->inflow : nullptr;
    a.lops = (j < p->l) ? p->lops : nullptr;
    a.ugrid = p->ugrid;
    a.gtarg = p->gtarg;
    a.shard_end = (p->shard && j < p->l) ? 1 : 0;
    return a;
}

// kernels per marginal product in an iteration: carry scan + tile products
// (three-phase, l <= 5), or 2 (NB levels x contribution + scan) + products
int launches_per_product(mmot_plan p) { return p->three_phase ? 2 : 2 * ((p->NB + 1) / 2 + p->NB) + 2; }

// kernel ids: 2 k_tops, 3 k_carry, 4 k_tile (three-phase design, l <= 5);
// 5 k_wpass, 6 k_lscan, 4 k_wprod (level passes and warp tiles, l >= 6);
// 0, 1 are not used by marginal products (objective sweeps only)
mmot_status timed_launch(mmot_plan p, int kernel, const SweepArgs &a, bool fp64, int SL = 0, int fwd = 0)
{
    p->launches += 1;
    auto go = [&]() -> cudaError_t {
        if (p->NB > kMaxOpBits) return launch_levels(p->NB, a, fp64, p->st, kernel, SL, fwd);
        return launch_ops(p->NB, a, fp64, p->st, kernel);
    };
    if (!p->profile) {
        CUDA_TRY(go());
        return MMOT_OK;
    }
    mmot_plan_s::Rec r;
    r.kernel = kernel;
    CUDA_TRY(cudaEventCreate(&r.a));
    CUDA_TRY(cudaEventCreate(&r.b));
    p->recs.push_back(r);
    CUDA_TRY(cudaEventRecord(r.a, p->st));
    CUDA_TRY(go());
    CUDA_TRY(cudaEventRecord(r.b, p->st));
    return MMOT_OK;
}

// One marginal product for target j.  Look-back design: backward scan, then
// forward scan with combine and epilogue.  Three-phase design: tile operators
// (only if the current ones belong to another target), carry scan, then the
// tile products; after an update the same launch computes the operators of
// target jnext from the new potentials.
mmot_status enqueue_product(mmot_plan p, int j, int mode, double *out, int jnext = -1)
{
    SweepArgs a = make_args(p, j, mode, out);
    const bool fp64 = (p->prec == MMOT_FP64);
    if (p->three_phase) {
        mmot_status s;
        // batches: tiles of frozen instances skip the fused operator update, so
        // products that read every tile start from fresh operators
        const bool all_tiles = (p->batch && mode != MODE_UPDATE && mode != MODE_RESIDUAL);
        if (p->ops_target != j || all_tiles) {
            s = timed_launch(p, 2, a, fp64);
            if (s != MMOT_OK) return s;
            p->ops_target = j;
        }
        CUDA_TRY(cudaMemsetAsync(p->cflags, 0, sizeof(int) * p->cflags_n, p->st));
        s = timed_launch(p, 3, a, fp64);
        if (s != MMOT_OK) return s;
        a.jnext = (mode == MODE_UPDATE) ? jnext : -1;
        s = timed_launch(p, 4, a, fp64);
        if (s != MMOT_OK) return s;
        if (a.jnext >= 0) p->ops_target = a.jnext;
        return MMOT_OK;
    }
    // level passes: backward and forward carries two levels per walk (the
    // pass of level lv also gives level lv+1 its share that does not go
    // through a level-lv carry), one scan per level, then the tile products
    // with both carries known
    CUDA_TRY(cudaMemsetAsync(p->cflags, 0, sizeof(int) * p->cflags_n, p->st));
    a.coef = p->coef;
    for (int fwd = 0; fwd < 2; ++fwd) {
        for (int lv = 1; lv <= p->NB; lv += 2) {
            const bool pair = (lv + 1 <= p->NB);
            a.pair = pair ? 1 : 0;
            mmot_status s = timed_launch(p, 5, a, fp64, lv, fwd);
            if (s != MMOT_OK) return s;
            a.pair = 0;
            s = timed_launch(p, 6, a, fp64, lv, fwd);
            if (s != MMOT_OK) return s;
            if (pair) {
                a.pair = 1;
                s = timed_launch(p, 6, a, fp64, lv + 1, fwd);
                if (s != MMOT_OK) return s;
            }
        }
    }
    a.pair = 0;
    mmot_status s = timed_launch(p, 7, a, fp64);
    if (s != MMOT_OK) return s;
    return timed_launch(p, 4, a, fp64);
}

template <int Lm>
cudaError_t launch_obj_l(const SweepArgs &a, bool fp64, cudaStream_t st, int kind)
{
    return fp64 ? launch_objective<Lm, double>(a, st, kind) : launch_objective<Lm, float>(a, st, kind);
}

cudaError_t launch_obj(int l, const SweepArgs &a, bool fp64, cudaStream_t st, int kind)
{
    switch (l) {
    case 2: return launch_obj_l<2>(a, fp64, st, kind);
    case 3: return launch_obj_l<3>(a, fp64, st, kind);
    case 4: return launch_obj_l<4>(a, fp64, st, kind);
    case 5: return launch_obj_l<5>(a, fp64, st, kind);
    case 6: return launch_obj_l<6>(a, fp64, st, kind);
    case 7: return launch_obj_l<7>(a, fp64, st, kind);
    default: return cudaErrorInvalidValue;   // l = 8: warp tiles (launch_objective_warp8)
    }
}

mmot_status ensure_objective_scratch(mmot_plan p)
{
    if (p->obj_ready) return MMOT_OK;
    const int l = p->l;
    const size_t nt = (size_t)p->nt, ns = (size_t)1 << l, sf = p->sfsz;
    CUDA_TRY(p->alloc(&p->o_bc, nt * ns * sf));
    CUDA_TRY(p->alloc(&p->o_lnz, nt));
    if (l == 8) {
        // warp tiles: level passes and per-state scans, then the objective kernel
        CUDA_TRY(p->alloc(&p->o_fc, nt * ns * sf));
        CUDA_TRY(p->alloc(&p->o_agg, nt * ns * sf));
        CUDA_TRY(p->alloc(&p->o_decF, p->h_odecF.size()));
        CUDA_TRY(p->alloc(&p->o_decB, p->h_odecB.size()));
        CUDA_TRY(p->alloc(&p->o_cflags, (size_t)2 * ns * 32));
        CUDA_TRY(p->alloc(&p->o_cagg, (size_t)2 * ns * 32 * sf));
        CUDA_TRY(p->alloc(&p->o_coef, nt * (size_t)l * sf));
        CUDA_TRY(cudaMemcpyAsync(p->o_decF, p->h_odecF.data(), p->h_odecF.size(), cudaMemcpyHostToDevice, p->st));
        CUDA_TRY(cudaMemcpyAsync(p->o_decB, p->h_odecB.data(), p->h_odecB.size(), cudaMemcpyHostToDevice, p->st));
        CUDA_TRY(cudaMemsetAsync(p->o_fc, 0, nt * ns * sf, p->st));
        CUDA_TRY(cudaMemsetAsync(p->o_bc, 0, nt * ns * sf, p->st));
    } else if (l <= kMaxOpBits) {
        CUDA_TRY(p->alloc(&p->o_fc, nt * ns * sf));
        CUDA_TRY(p->alloc(&p->o_opF, nt * l * ns * sf));
        CUDA_TRY(p->alloc(&p->o_opB, nt * l * ns * sf));
        CUDA_TRY(p->alloc(&p->o_decF, p->h_odecF.size()));
        CUDA_TRY(p->alloc(&p->o_decB, p->h_odecB.size()));
        CUDA_TRY(p->alloc(&p->o_cflags, (size_t)2 * 32 * (l + 1)));
        CUDA_TRY(p->alloc(&p->o_cagg, (size_t)2 * 32 * ns * sf));
        CUDA_TRY(cudaMemcpyAsync(p->o_decF, p->h_odecF.data(), p->h_odecF.size(), cudaMemcpyHostToDevice, p->st));
        CUDA_TRY(cudaMemcpyAsync(p->o_decB, p->h_odecB.data(), p->h_odecB.size(), cudaMemcpyHostToDevice, p->st));
    } else {
        CUDA_TRY(p->alloc(&p->o_agg, nt * ns * sf));
        CUDA_TRY(p->alloc(&p->o_inc, nt * ns * sf));
        p->o_flags_bytes = sizeof(int) * (nt * (l + 1) + 1);
        CUDA_TRY(p->alloc(&p->o_flags, nt * (l + 1) + 1));
    }
    p->obj_ready = true;
    return MMOT_OK;
}

// W = <C, T> by the gap formula (objective.cuh): per-tile W/Z into
// p->partial, their sum into p->dsum[0], ln Z of every tile into p->o_lnz.
mmot_status enqueue_cost(mmot_plan p)
{
    mmot_status s = ensure_objective_scratch(p);
    if (s != MMOT_OK) return s;
    const int l = p->l;
    const bool fp64 = (p->prec == MMOT_FP64);
    SweepArgs a = make_args(p, l, MODE_OUT_M, p->o_lnz);
    a.agg = p->o_agg;
    a.inc = p->o_inc;
    a.flags = p->o_flags;
    a.counter = p->o_flags ? p->o_flags + (size_t)p->nt * (l + 1) : nullptr;
    a.bcarry = p->o_bc;
    a.fcarry = p->o_fc;
    a.opF = p->o_opF;
    a.opB = p->o_opB;
    a.pdecF = p->o_decF;
    a.pdecB = p->o_decB;
    a.cflags = p->o_cflags;
    a.cagg = p->o_cagg;
    if (l == 8) {
        // two levels per walk, as in the products: the pass of level lv also
        // gives level lv+1 its own share and the coefficients of the share
        // that goes through a level-lv carry
        CUDA_TRY(cudaMemsetAsync(p->o_cflags, 0, sizeof(int) * 2 * 256 * 32, p->st));
        a.coef = p->o_coef;
        auto lo = [&](int kind, int lv, int fwd) {
            return fp64 ? launch_objective_warp8<double>(a, p->st, kind, lv, fwd)
                        : launch_objective_warp8<float>(a, p->st, kind, lv, fwd);
        };
        for (int fwd = 0; fwd < 2; ++fwd) {
            for (int lv = 1; lv <= l; lv += 2) {
                const bool pair = (lv + 1 <= l);
                a.pair = pair ? 1 : 0;
                CUDA_TRY(lo(5, lv, fwd));
                a.pair = 0;
                CUDA_TRY(lo(6, lv, fwd));
                p->launches += 2;
                if (pair) {
                    a.pair = 1;
                    CUDA_TRY(lo(6, lv + 1, fwd));
                    p->launches += 1;
                }
            }
        }
        a.pair = 0;
        CUDA_TRY(fp64 ? launch_objective_warp8<double>(a, p->st, 7, 0, 0)
                      : launch_objective_warp8<float>(a, p->st, 7, 0, 0));
    } else if (l <= kMaxOpBits) {
        CUDA_TRY(launch_obj(l, a, fp64, p->st, 2));
        CUDA_TRY(cudaMemsetAsync(p->o_cflags, 0, sizeof(int) * 2 * 32 * (l + 1), p->st));
        CUDA_TRY(launch_obj(l, a, fp64, p->st, 3));
        CUDA_TRY(launch_obj(l, a, fp64, p->st, 5));
    } else {
        CUDA_TRY(cudaMemsetAsync(p->o_flags, 0, p->o_flags_bytes, p->st));
        CUDA_TRY(launch_obj(l, a, fp64, p->st, 0));
        CUDA_TRY(cudaMemsetAsync(p->o_flags, 0, p->o_flags_bytes, p->st));
        CUDA_TRY(launch_obj(l, a, fp64, p->st, 5));
    }
    k_sum_partials<<<1, 256, 0, p->st>>>(p->partial, p->nt, p->dsum, 0);
    CUDA_TRY(cudaGetLastError());
    p->launches += (l == 8) ? 1 : ((l <= kMaxOpBits) ? 4 : 3);
    return MMOT_OK;
}

// g_k = -eps ln N_k, beta = -ln N_k, lphi = 0
__global__ void k_reset(double *g, int64_t n, double v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        g[i] = v;
}

// x[i] = v for i < n (the scaled phi of the tile kernels after a reset)
template <typename Tv>
__global__ void k_fill(Tv *x, int64_t n, Tv v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

// g_k of instance q (one block per instance) = its initial value
__global__ void k_reset_seg(double *g, const int64_t *off, const double *g0, int k, int l)
{
    const int q = blockIdx.x;
    const int64_t i0 = off[(size_t)q * l + k], i1 = off[(size_t)(q + 1) * l + k];
    const double v = g0[(size_t)q * l + k];
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) g[i] = v;
}

// Objective sums of instance q (one block each), compensated (Kahan) over
// the instance's tiles: from part4 (per tile: plan-marginal mass, L1 error,
// sum g marg, sum g mu of one marginal) into acc[q*5 + 0..3] (the mass is
// set, the others accumulate over the marginals), or, with w_lnz, the
// transport cost W = Z * sum of the per-tile W_b / Z_b (partial) into
// acc[q*5 + 4], Z from ln Z of the instance's first tile.
__global__ void k_seg_obj(const double *part4, const double *partial, const double *w_lnz, const int32_t *t0,
                          double *acc, int set_mass, int stop)
{
    const int q = blockIdx.x;
    const int b0 = t0[q], b1 = t0[q + 1];
    const int NQ = w_lnz ? 1 : 4;
    __shared__ double s_s[4][256], s_c[4][256];
    for (int m = 0; m < NQ; ++m) {
        double sum = 0.0, c = 0.0;
        for (int b = b0 + (int)threadIdx.x; b < b1; b += blockDim.x) {
            const double y = (w_lnz ? partial[b] : part4[(size_t)b * 4 + m]) - c;
            const double t = sum + y;
            c = (t - sum) - y;
            sum = t;
        }
        s_s[m][threadIdx.x] = sum;
        s_c[m][threadIdx.x] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int m = 0; m < NQ; ++m) {
            double S = 0.0, Cc = 0.0;
            for (int i = 0; i < (int)blockDim.x; ++i) {
                const double y = s_s[m][i] - s_c[m][i] - Cc;
                const double t = S + y;
                Cc = (t - S) - y;
                S = t;
            }
            if (w_lnz) {
                const double lz = w_lnz[b0];
                acc[(size_t)q * 6 + 4] = (lz == -INFINITY) ? 0.0 : S * exp(lz);
            } else if (m == 0) {
                if (set_mass) acc[(size_t)q * 6 + 0] = S;
            } else {
                acc[(size_t)q * 6 + m] += S;
                if (m == 1 && stop) acc[(size_t)q * 6 + 5] += S;
            }
        }
    }
}

// res[q] (+)= sum of the per-tile partial sums of instance q (one thread per
// instance, compensated)
__global__ void k_seg_sum(const double *partial, const int32_t *t0, int nseg, double *res, int accumulate)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nseg) return;
    double sum = 0.0, c = 0.0;
    for (int b = t0[q]; b < t0[q + 1]; ++b) {
        const double y = partial[b] - c;
        const double t = sum + y;
        c = (t - sum) - y;
        sum = t;
    }
    res[q] = accumulate ? res[q] + sum : sum;
}

// One Gauss-Seidel iteration.  In the three-phase design it expects the tile
// operators of target 0 to be current and leaves them current.
mmot_status enqueue_iteration(mmot_plan p)
{
    for (int j = 0; j < p->l; ++j) {
        mmot_status s = enqueue_product(p, j, MODE_UPDATE, nullptr, (j + 1) % p->l);
        if (s != MMOT_OK) return s;
    }
    return MMOT_OK;
}

mmot_status ensure_ops(mmot_plan p, int j)
{
    if (!p->three_phase || p->ops_target == j) return MMOT_OK;
    SweepArgs a = make_args(p, j, MODE_UPDATE, nullptr);
    mmot_status s = timed_launch(p, 2, a, p->prec == MMOT_FP64);
    if (s == MMOT_OK) p->ops_target = j;
    return s;
}

mmot_status check_device_error(mmot_plan p)
{
    int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->st));
    CUDA_TRY(cudaStreamSynchronize(p->st));
    if (h) {
        CUDA_TRY(cudaMemsetAsync(p->err, 0, sizeof(int), p->st));
        // a wait also gives up (and sets the timeout bit) once another error
        // is recorded: report that error first
        if (h & ERR_RANGE) return fail(MMOT_ERR_RANGE, "a tile exceeded its target-point capacity");
        if (h & ERR_NONFINITE) return fail(MMOT_ERR_NONFINITE, "a potential became NaN or infinite");
        if (h & ERR_TIMEOUT) return fail(MMOT_ERR_TIMEOUT, "an inter-tile wait reached its poll limit");
    }
    return MMOT_OK;
}

// residual of marginals [k0, k1) into p->dsum[0]
mmot_status enqueue_residual(mmot_plan p, int k0, int k1)
{
    CUDA_TRY(cudaMemsetAsync(p->dsum, 0, sizeof(double), p->st));
    for (int k = k0; k < k1; ++k) {
        mmot_status s = enqueue_product(p, k, MODE_RESIDUAL, nullptr);
        if (s != MMOT_OK) return s;
        k_sum_partials<<<1, 256, 0, p->st>>>(p->partial, p->nt, p->dsum, 1);
        CUDA_TRY(cudaGetLastError());
        p->launches += 1;
    }
    return MMOT_OK;
}

mmot_status read_scalar(mmot_plan p, const double *d, double *h)
{
    CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(double), cudaMemcpyDeviceToHost, p->st));
    CUDA_TRY(cudaStreamSynchronize(p->st));
    return MMOT_OK;
}

// Re-centre the merged-order copy of ln phi_k after g_k changed on the host side.
// flag[0] |= 1 if some g[i] is NaN or +inf
__global__ void k_check_pot(const double *g, int64_t n, int *flag)
{
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = g[i];
        if (v != v || v == INFINITY) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// New potentials g_k (device) into the stream copies of phi_k: per tile the
// baseline beta = max of g/eps over the tile's points of marginal k (0 if
// none is finite), then ln phi - beta and (tile kernels) e^{g/eps - beta} at
// those points.  One block per tile; the tile's points of marginal k are
// ranked in merged order (local index = points of k before the tile + rank).
template <typename Tv>
__global__ void __launch_bounds__(256) k_recentre(const uint32_t *tstart, const uint8_t *mid, const int32_t *cnt,
                                                  const uint32_t *toff, int l, int k, double inv_eps,
                                                  const double *g, double *beta, Tv *lphi, Tv *ephi)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int b = blockIdx.x;
    const uint32_t t0 = tstart[b];
    const int n = (int)(tstart[b + 1] - t0);
    const int32_t off = cnt[(size_t)b * l + k];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    __shared__ int s_cnt[8];
    __shared__ double s_max[8];
    // rank of the point r among the tile's points of k, -1 if not of k
    auto walk = [&](auto &&fn) {
        int base = 0;
        for (int c0 = 0; c0 < n; c0 += 256) {
            const int r = c0 + tid;
            const bool hit = r < n && mid[t0 + r] == k;
            const unsigned bal = __ballot_sync(FULL, hit);
            __syncthreads();
            if (lane == 0) s_cnt[w] = __popc(bal);
            __syncthreads();
            int before = 0, tot = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = s_cnt[q];
                if (q < w) before += c;
                tot += c;
            }
            if (hit) fn(r, base + before + __popc(bal & ((1u << lane) - 1u)));
            base += tot;
        }
    };
    double mx = -INFINITY;
    walk([&](int, int rank) { mx = fmax(mx, g[off + rank] * inv_eps); });
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL, mx, o));
    if (lane == 0) s_max[w] = mx;
    __syncthreads();
    double bx = -INFINITY;
#pragma unroll
    for (int q = 0; q < 8; ++q) bx = fmax(bx, s_max[q]);
    if (!(bx > -INFINITY && bx < INFINITY)) bx = 0.0;
    if (tid == 0) beta[(size_t)b * l + k] = bx;
    walk([&](int r, int rank) {
        const double v = g[off + rank] * inv_eps - bx;
        lphi[t0 + r] = (Tv)v;
        if (ephi) ephi[toff[b] + r] = (v == -INFINITY) ? Tv(0) : (Tv)exp(v);
    });
}

mmot_status upload_potential(mmot_plan p, int k, const std::vector<double> &g)
{
    const int l = p->l;
    const int nt = p->nt;
    // 1/eps of every point of marginal k: each instance of a batch has its own eps
    std::vector<double> ie((size_t)p->N[k], 1.0 / p->eps);
    if (p->nseg > 1 && p->seg_off.size() == (size_t)(p->nseg + 1) * l)
        for (int q = 0; q < p->nseg; ++q)
            for (int64_t i = p->seg_off[(size_t)q * l + k]; i < p->seg_off[(size_t)(q + 1) * l + k]; ++i)
                ie[(size_t)i] = 1.0 / p->seg_eps[q];
    std::vector<double> bmax(nt, -INFINITY);
    for (int64_t i = 0; i < p->N[k]; ++i) {
        const uint32_t t = p->h_mpos[k][i];
        const uint32_t b = p->h_tile_of[t];
        bmax[b] = std::max(bmax[b], g[i] * ie[i]);
    }
    for (int b = 0; b < nt; ++b) {
        double v = bmax[b];
        if (!std::isfinite(v)) v = 0.0;
        p->h_beta[(size_t)b * l + k] = v;
    }
    // lphi for the points of marginal k, written as one full upload of lphi
    std::vector<unsigned char> lp((size_t)p->T * p->esz);
    CUDA_TRY(cudaMemcpyAsync(lp.data(), p->lphi, lp.size(), cudaMemcpyDeviceToHost, p->st));
    CUDA_TRY(cudaStreamSynchronize(p->st));
    for (int64_t i = 0; i < p->N[k]; ++i) {
        const uint32_t t = p->h_mpos[k][i];
        const uint32_t b = p->h_tile_of[t];
        const double v = g[i] * ie[i] - p->h_beta[(size_t)b * l + k];
        if (p->esz == 8)
            reinterpret_cast<double *>(lp.data())[t] = v;
        else
            reinterpret_cast<float *>(lp.data())[t] = (float)v;
    }
    // the same points in the padded stream of the tile kernels: e^{g/eps - beta}
    std::vector<unsigned char> ep;
    if (p->three_phase) {
        ep.resize((size_t)p->Tpad * p->esz);
        CUDA_TRY(cudaMemcpyAsync(ep.data(), p->ephi, ep.size(), cudaMemcpyDeviceToHost, p->st));
        CUDA_TRY(cudaStreamSynchronize(p->st));
        for (int64_t i = 0; i < p->N[k]; ++i) {
            const uint32_t t = p->h_mpos[k][i];
            const uint32_t b = p->h_tile_of[t];
            const size_t u = (size_t)p->h_toff[b] + (t - p->h_tstart[b]);
            const double v = std::exp(g[i] * ie[i] - p->h_beta[(size_t)b * l + k]);
            if (p->esz == 8)
                reinterpret_cast<double *>(ep.data())[u] = v;
            else
                reinterpret_cast<float *>(ep.data())[u] = (float)v;
        }
    }
    // the device beta of other marginals may have moved: read them back first
    std::vector<double> hb((size_t)nt * l);
    CUDA_TRY(cudaMemcpyAsync(hb.data(), p->beta, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, p->st));
    CUDA_TRY(cudaStreamSynchronize(p->st));
    for (int b = 0; b < nt; ++b) hb[(size_t)b * l + k] = p->h_beta[(size_t)b * l + k];
    CUDA_TRY(cudaMemcpyAsync(p->beta, hb.data(), sizeof(double) * hb.size(), cudaMemcpyHostToDevice, p->st));
    CUDA_TRY(cudaMemcpyAsync(p->lphi, lp.data(), lp.size(), cudaMemcpyHostToDevice, p->st));
    if (p->three_phase) CUDA_TRY(cudaMemcpyAsync(p->ephi, ep.data(), ep.size(), cudaMemcpyHostToDevice, p->st));
    CUDA_TRY(cudaMemcpyAsync(p->g[k], g.data(), sizeof(double) * p->N[k], cudaMemcpyHostToDevice, p->st));
    CUDA_TRY(cudaStreamSynchronize(p->st));
    p->ops_target = -1;
    return MMOT_OK;
}

// Plan of one instance, or of a batch of independent instances with the same
// l laid out one after the other (tiles never straddle two instances).
// tiles one carry scan handles (k_carry: 32 chunks x 256 threads x 8 tiles)
constexpr int kMaxCarryTiles = 32 * 256 * 8;

mmot_status plan_build(int l, const std::vector<InstanceIn> &ins, mmot_precision prec, int inputs_on_device,
                       void *cuda_stream, mmot_plan *out, int tile_points = 0, bool batch = false)
{
    *out = nullptr;
    if (prec != MMOT_FP64 && prec != MMOT_FP32_SCAN_FP64_POT)
        return fail(MMOT_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    const int nin = (int)ins.size();
    if (nin < 1) return fail(MMOT_ERR_INVALID_ARG, "no instance");
    int64_t T = 0;
    int64_t N[MMOT_MAXL] = {0};
    for (int q = 0; q < nin; ++q) {
        const InstanceIn &in = ins[q];
        if (!(in.eps > 0.0) || !std::isfinite(in.eps))
            return fail(MMOT_ERR_INVALID_ARG, "instance %d: eps must be positive and finite", q);
        for (int k = 0; k < l; ++k) {
            if (in.N[k] < 1) return fail(MMOT_ERR_INVALID_ARG, "instance %d: N[%d] = %lld < 1", q, k, (long long)in.N[k]);
            if (!in.x[k] || !in.mu[k]) return fail(MMOT_ERR_INVALID_ARG, "instance %d: x[%d] or mu[%d] is NULL", q, k, k);
            T += in.N[k];
            N[k] += in.N[k];
        }
    }
    if (T >= (int64_t)1 << 31) return fail(MMOT_ERR_RANGE, "sum N = %lld too large", (long long)T);
    const double eps = ins[0].eps;

    // ---- inputs to host, validation, per-instance layouts (layout.h) --------
    const bool fp64 = (prec == MMOT_FP64);
    int K = 0, NT = 0, jcap = 0;
    shape_of(l - 1, fp64, &K, &NT, &jcap);
    if (l - 1 <= kMaxOpBits) jcap = tile_jcap(l - 1, fp64);   // the tile kernels' target capacity
    if (l - 1 > kMaxOpBits) {
        // warp-tile products (warp.cuh)
        K = fp64 ? wshape_k<double>(l - 1) : wshape_k<float>(l - 1);
        jcap = K / 4;   // WShape<NB, V>::JCAP
    }
    if (tile_points > 0) K = std::max(32, std::min(K, tile_points));
    const double limit = fp64 ? kSpanLimitF64 : kSpanLimitF32;
    double ugrid_h = 0.0;   // > 0: one uniform grid of step ugrid_h for every marginal
    HostLayout L;
    L.l = l;
    std::vector<HVec<double>> hmu(l);
    std::vector<int32_t> hseg;
    std::vector<double> hteps;
    std::vector<int32_t> seg_tile0(1, 0);
    std::vector<int64_t> seg_off((size_t)(nin + 1) * l, 0);   // first local index of instance q in marginal k
    for (int q = 0; q < nin; ++q) {
        const InstanceIn &in = ins[q];
        std::vector<HVec<double>> hx(l), qmu(l);
        int64_t Tq = 0;
        for (int k = 0; k < l; ++k) {
            const int64_t n = in.N[k];
            Tq += n;
            hx[k].resize(n);
            qmu[k].resize(n);
            if (inputs_on_device) {
                CUDA_TRY(cudaMemcpy(hx[k].data(), in.x[k], sizeof(double) * n, cudaMemcpyDeviceToHost));
                CUDA_TRY(cudaMemcpy(qmu[k].data(), in.mu[k], sizeof(double) * n, cudaMemcpyDeviceToHost));
            }
        }
        if (!inputs_on_device) {
            // host inputs: plain copies, one host thread per marginal for large inputs
            auto copy_marginal = [&](int k) {
                std::memcpy(hx[k].data(), in.x[k], sizeof(double) * in.N[k]);
                std::memcpy(qmu[k].data(), in.mu[k], sizeof(double) * in.N[k]);
            };
            if (layout_threads(Tq) > 1)
                host_parallel(l, copy_marginal);
            else
                for (int k = 0; k < l; ++k) copy_marginal(k);
        }
        // checks of the marginals (one host thread each for large inputs);
        // the first failure in marginal order is reported
        std::vector<mmot_status> kst(l, MMOT_OK);
        std::vector<std::string> kmsg(l);
        auto check_marginal = [&](int k) {
            const int64_t n = in.N[k];
            char buf[160];
            const HVec<double> &xk = hx[k], &mk = qmu[k];
            for (int64_t i = 0; i < n; ++i) {
                if (!std::isfinite(xk[i])) {
                    std::snprintf(buf, sizeof(buf), "instance %d: x[%d][%lld] not finite", q, k, (long long)i);
                    kst[k] = MMOT_ERR_INVALID_ARG;
                    kmsg[k] = buf;
                    return;
                }
                if (i > 0 && xk[i] < xk[i - 1]) {
                    std::snprintf(buf, sizeof(buf), "instance %d: x[%d] decreases at index %lld", q, k, (long long)i);
                    kst[k] = MMOT_ERR_UNSORTED;
                    kmsg[k] = buf;
                    return;
                }
            }
            // compensated (Neumaier) sum: error about one rounding of the
            // total, far inside the 1e-12 check (a long double sum is
            // software quad precision on some hosts)
            double sum = 0.0, comp = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                const double m = mk[i];
                if (!(m >= 0.0) || !std::isfinite(m)) {
                    std::snprintf(buf, sizeof(buf), "instance %d: mu[%d][%lld] negative or not finite", q, k,
                                  (long long)i);
                    kst[k] = MMOT_ERR_INVALID_ARG;
                    kmsg[k] = buf;
                    return;
                }
                const double t = sum + m;
                comp += (std::fabs(sum) >= std::fabs(m)) ? (sum - t) + m : (m - t) + sum;
                sum = t;
            }
            sum += comp;
            if (!in.Ntot && std::fabs(sum - 1.0) > 1e-12) {
                std::snprintf(buf, sizeof(buf), "instance %d: mu[%d] sums to %.17g, not 1", q, k, sum);
                kst[k] = MMOT_ERR_INVALID_ARG;
                kmsg[k] = buf;
            }
        };
        if (layout_threads(Tq) > 1)
            host_parallel(l, check_marginal);
        else
            for (int k = 0; k < l; ++k) check_marginal(k);
        for (int k = 0; k < l; ++k)
            if (kst[k] != MMOT_OK) return fail(kst[k], "%s", kmsg[k].c_str());
        for (int k = 0; k < l; ++k) {
            const int64_t n = in.N[k];
            if (hmu[k].empty())
                hmu[k] = std::move(qmu[k]);
            else
                hmu[k].insert(hmu[k].end(), qmu[k].begin(), qmu[k].end());
            seg_off[(size_t)(q + 1) * l + k] = seg_off[(size_t)q * l + k] + n;
        }
        if (nin == 1) {
            // one uniform grid for every marginal: identical coordinates,
            // x_i = x_0 + i h within 1e-9 h (tile kernels, l <= 5)
            bool u = (l - 1 <= kMaxOpBits) && in.N[0] >= 2;
            for (int k = 1; k < l && u; ++k) u = (in.N[k] == in.N[0]) && (hx[k] == hx[0]);
            double h = 0.0;
            if (u) {
                const int64_t n = in.N[0];
                h = (hx[0][n - 1] - hx[0][0]) / (double)(n - 1);
                u = h > 0.0;
                for (int64_t i = 0; i < n && u; ++i)
                    u = std::fabs(hx[0][i] - (hx[0][0] + (double)i * h)) <= 1e-9 * h;
            }
            ugrid_h = u ? h : 0.0;
        }
        HostLayout Lq;
        build_layout(l, in.N, hx, in.eps, K, jcap, limit, Lq);
        const int ntq = Lq.nt;
        if (q == 0)
            L = std::move(Lq);   // the first instance: appending to an empty layout is the layout itself
        else
            append_layout(L, Lq, &seg_off[(size_t)q * l]);
        for (int b = 0; b < ntq; ++b) {
            hseg.push_back(q);
            hteps.push_back(in.eps);
        }
        seg_tile0.push_back(L.nt);
    }

    if (l - 1 <= kMaxOpBits && L.nt > kMaxCarryTiles)
        return fail(MMOT_ERR_RANGE, "%d tiles exceed the carry scan's %d", L.nt, kMaxCarryTiles);
    mmot_plan p = new (std::nothrow) mmot_plan_s();
    if (!p) return fail(MMOT_ERR_OOM, "host allocation failed");
    p->l = l;
    p->T = T;
    p->eps = eps;
    p->prec = (int)prec;
    for (int k = 0; k < l; ++k) p->N[k] = N[k];
    p->shard = (nin == 1 && ins[0].Ntot != nullptr);
    for (int k = 0; k < l; ++k) p->Ninit[k] = (int64_t)ins[0].init_count(k);
    p->NB = l - 1;
    p->NS = 1 << p->NB;
    p->K = K;
    p->NT = NT;
    p->nseg = nin;
    p->batch = batch;
    p->seg_tile0 = seg_tile0;
    p->seg_off = seg_off;
    for (int q = 0; q < nin; ++q) {
        p->seg_eps.push_back(ins[q].eps);
        for (int k = 0; k < l; ++k) p->seg_N.push_back(ins[q].N[k]);
    }
    if (cuda_stream) {
        p->st = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete p;
            return fail(MMOT_ERR_CUDA, "stream creation failed: %s", cudaGetErrorString(e));
        }
        p->own_stream = true;
    }

    // ---- merged order and tiles ----------------------------------------------
    const int nt = L.nt;
    p->nt = nt;
    // the layout's arrays move into the plan (the layout is not read again)
    p->h_mid = std::move(L.mid);
    for (int k = 0; k < l; ++k) p->h_mpos[k] = std::move(L.mpos[k]);
    p->h_tstart = std::move(L.tstart);
    p->h_tile_of = std::move(L.tile_of);
    p->h_reftile = std::move(L.reftile);
    std::vector<uint32_t> &ts = p->h_tstart;
    std::vector<double> &hspan = L.span;
    HVec<double> &hpos = L.pos;
    std::vector<int32_t> &hcnt = L.cnt, &href = p->h_reftile;
    // initial baselines: g_k = -eps ln N_k of the tile's instance
    p->h_beta0.assign((size_t)nt * l, 0.0);
    for (int b = 0; b < nt; ++b)
        for (int k = 0; k < l; ++k)
            p->h_beta0[(size_t)b * l + k] = -std::log(ins[hseg[b]].init_count(k));
    p->h_beta = p->h_beta0;

    // ---- device allocation and upload -------------------------------------
#define PA(ptr, n)                                          \
    do {                                                    \
        cudaError_t e_ = p->alloc(&ptr, (size_t)(n));       \
        if (e_ != cudaSuccess) {                            \
            delete p;                                       \
            return fail(MMOT_ERR_OOM, "cudaMalloc %s", #ptr); \
        }                                                   \
    } while (0)
    p->esz = fp64 ? 8 : 4;
    {
        unsigned char *q1 = nullptr, *q2 = nullptr;
        PA(q1, (size_t)T * p->esz);
        PA(q2, (size_t)T * p->esz);
        p->pos = q1;
        p->lphi = q2;
    }
    PA(p->mid, T);
    PA(p->tstart, nt + 1);
    PA(p->ulb, nt);
    PA(p->urb, nt);
    PA(p->span, nt);
    PA(p->cnt, (size_t)nt * l);
    PA(p->reftile, (size_t)nt * l);
    PA(p->beta, (size_t)nt * l);
    int64_t maxN = 1;
    for (int k = 0; k < l; ++k) {
        PA(p->g[k], N[k]);
        PA(p->lnmu[k], N[k]);
        PA(p->mu[k], N[k]);
        maxN = std::max(maxN, N[k]);
    }
    p->sfsz = fp64 ? 16 : 8;
    PA(p->agg, (size_t)nt * p->NS * p->sfsz);
    PA(p->inc, (size_t)nt * p->NS * p->sfsz);
    PA(p->bcarry, (size_t)nt * p->NS * p->sfsz);
    p->three_phase = (p->NB <= kMaxOpBits);
    PA(p->fcarry, (size_t)nt * p->NS * p->sfsz);
    PA(p->pdecF, (size_t)nt * (p->NB + 1) * p->sfsz);
    PA(p->pdecB, (size_t)nt * (p->NB + 1) * p->sfsz);
    // chunk flags / contributions: [2][32][NB+1] (three-phase scan) or
    // [2][NS][32] (one scalar scan per state, level passes)
    p->cflags_n = p->three_phase ? (size_t)2 * 32 * (p->NB + 1) : (size_t)2 * p->NS * 32;
    PA(p->cflags, p->cflags_n);
    PA(p->cagg, (size_t)2 * 32 * p->NS * p->sfsz);
    if (!p->three_phase) {
        PA(p->coef, (size_t)nt * p->NB * p->sfsz);
        unsigned char *gt = nullptr;
        int64_t mx = 1;
        for (int k = 0; k < l; ++k) mx = std::max(mx, N[k]);
        PA(gt, (size_t)mx * p->NS * p->sfsz);
        p->gtarg = gt;
    }
    if (p->shard) {
        PA(p->inflow, (size_t)2 * p->NS * p->sfsz);
        PA(p->d_lnop, (size_t)2 * (p->NB + 1) * p->NS);
    }
    if (p->three_phase) {
        PA(p->opF, (size_t)nt * p->NB * p->NS * p->sfsz);
        PA(p->opB, (size_t)nt * p->NB * p->NS * p->sfsz);
        {
            unsigned char *lo = nullptr;
            PA(lo, (size_t)nt * tile_lops_bytes(p->NB, fp64));
            p->lops = lo;
        }
        // padded stream: every tile starts on a 16-element boundary
        p->h_toff.resize(nt);
        int64_t o = 0;
        for (int b = 0; b < nt; ++b) {
            p->h_toff[b] = (uint32_t)o;
            o += ((int64_t)(ts[b + 1] - ts[b]) + 15) / 16 * 16;
        }
        p->Tpad = std::max<int64_t>(o, 16);
        if (p->Tpad >= ((int64_t)1 << 32)) {
            delete p;
            return fail(MMOT_ERR_RANGE, "padded stream too long");
        }
        PA(p->toff, nt);
        unsigned char *q1 = nullptr, *q2 = nullptr;
        if (ugrid_h > 0.0) {
            PA(q1, (size_t)(K / l + 2) * p->esz);   // grid steps within one tile
            p->ugrid = q1;
        } else {
            PA(q1, (size_t)p->Tpad * p->esz);
            p->epos = q1;
            PA(p->emid, p->Tpad);
        }
        PA(q2, (size_t)p->Tpad * p->esz);
        p->ephi = q2;
        if (!fp64)
            for (int k = 0; k < l; ++k) PA(p->lnmu_ff[k], N[k]);
    }
    PA(p->partial, nt);
    PA(p->part4, (size_t)nt * 4);
    PA(p->d_obj, (size_t)nin * 6);
    if (!batch) PA(p->d_segt0, 2);
    p->flags_bytes = sizeof(int) * ((size_t)nt * (p->NB + 1) + 1);
    PA(p->flags, (size_t)nt * (p->NB + 1) + 1);
    PA(p->err, 1);
    PA(p->dsum, 8);
    PA(p->scratch, maxN);
    if (batch) {
        PA(p->d_seg, nt);
        PA(p->d_teps, nt);
        PA(p->d_frozen, nin);
        PA(p->d_segt0, nin + 1);
        PA(p->d_res, nin);
        PA(p->d_goff, (size_t)(nin + 1) * l);
        PA(p->d_g0, (size_t)nin * l);
    }
#undef PA

    auto up = [&](void *d, const void *h, size_t bytes) {
        return cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, p->st);
    };
    HVec<unsigned char> hposb((size_t)T * p->esz);
    if (fp64)
        convert_parallel(T, hpos.data(), reinterpret_cast<double *>(hposb.data()));
    else
        convert_parallel(T, hpos.data(), reinterpret_cast<float *>(hposb.data()));
    cudaError_t ce = cudaSuccess;
    ce = ce ? ce : up(p->pos, hposb.data(), hposb.size());
    ce = ce ? ce : up(p->mid, p->h_mid.data(), T);
    ce = ce ? ce : cudaMemsetAsync(p->lphi, 0, (size_t)T * p->esz, p->st);   // ln phi = 0
    ce = ce ? ce : up(p->tstart, ts.data(), sizeof(uint32_t) * (nt + 1));
    std::vector<double> &hulb = L.ulb, &hurb = L.urb;
    ce = ce ? ce : up(p->ulb, hulb.data(), sizeof(double) * nt);
    ce = ce ? ce : up(p->urb, hurb.data(), sizeof(double) * nt);
    // exp(-w_s d) from each tile base to the next base in processing order
    std::vector<unsigned char> hdecF, hdecB;
    const std::vector<int32_t> segv = batch ? hseg : std::vector<int32_t>();
    if (l <= kMaxOpBits || l == 8) decay_tables(L, l, fp64, p->h_odecF, p->h_odecB, segv);
    decay_tables(L, p->NB, fp64, hdecF, hdecB, segv, p->shard);
    ce = ce ? ce : up(p->pdecF, hdecF.data(), hdecF.size());
    ce = ce ? ce : up(p->pdecB, hdecB.data(), hdecB.size());
    ce = ce ? ce : up(p->span, hspan.data(), sizeof(double) * nt);
    ce = ce ? ce : up(p->cnt, hcnt.data(), sizeof(int32_t) * nt * l);
    ce = ce ? ce : up(p->reftile, href.data(), sizeof(int32_t) * nt * l);
    ce = ce ? ce : up(p->beta, p->h_beta.data(), sizeof(double) * nt * l);
    std::vector<std::vector<double>> hg(l), hlm(l);
    for (int k = 0; k < l && ce == cudaSuccess; ++k) {
        hg[k].resize(N[k]);
        for (int q = 0; q < nin; ++q) {
            const double g0 = -ins[q].eps * std::log(ins[q].init_count(k));
            for (int64_t i = seg_off[(size_t)q * l + k]; i < seg_off[(size_t)(q + 1) * l + k]; ++i) hg[k][i] = g0;
        }
        hlm[k].resize(N[k]);
        {
            const int P = layout_threads(N[k]);
            const int64_t n = N[k];
            std::vector<double> &dst = hlm[k];
            const HVec<double> &src = hmu[k];
            host_parallel(P, [&](int pp) {
                for (int64_t i = n * pp / P; i < n * (pp + 1) / P; ++i) dst[i] = src[i] > 0 ? std::log(src[i]) : -INFINITY;
            });
        }
        ce = up(p->g[k], hg[k].data(), sizeof(double) * N[k]);
        ce = ce ? ce : up(p->lnmu[k], hlm[k].data(), sizeof(double) * N[k]);
        ce = ce ? ce : up(p->mu[k], hmu[k].data(), sizeof(double) * N[k]);
    }
    if (batch) {
        std::vector<double> g0((size_t)nin * l);
        for (int q = 0; q < nin; ++q)
            for (int k = 0; k < l; ++k) g0[(size_t)q * l + k] = -ins[q].eps * std::log(ins[q].init_count(k));
        ce = ce ? ce : up(p->d_seg, hseg.data(), sizeof(int32_t) * nt);
        ce = ce ? ce : up(p->d_teps, hteps.data(), sizeof(double) * nt);

        ce = ce ? ce : up(p->d_goff, seg_off.data(), sizeof(int64_t) * seg_off.size());
        ce = ce ? ce : up(p->d_g0, g0.data(), sizeof(double) * g0.size());
        ce = ce ? ce : cudaMemsetAsync(p->d_frozen, 0, sizeof(int32_t) * nin, p->st);
    }
    if (p->three_phase) {
        // padded stream: e^{pos}, scaled phi (1: lphi = 0), marginal (0xff: padding)
        const size_t Tp = (size_t)p->Tpad;
        const bool ug = (p->ugrid != nullptr);
        HVec<unsigned char> hep(ug ? 0 : Tp * p->esz), hph(Tp * p->esz);
        HVec<uint8_t> hem(ug ? 0 : Tp);
        if (fp64)
            fill_padded_stream<double>(nt, ts.data(), p->h_toff.data(), Tp, hpos.data(), p->h_mid.data(),
                                       ug ? nullptr : reinterpret_cast<double *>(hep.data()),
                                       reinterpret_cast<double *>(hph.data()), ug ? nullptr : hem.data());
        else
            fill_padded_stream<float>(nt, ts.data(), p->h_toff.data(), Tp, hpos.data(), p->h_mid.data(),
                                      ug ? nullptr : reinterpret_cast<float *>(hep.data()),
                                      reinterpret_cast<float *>(hph.data()), ug ? nullptr : hem.data());
        ce = ce ? ce : up(p->toff, p->h_toff.data(), sizeof(uint32_t) * nt);
        std::vector<unsigned char> hug;
        if (ug) {
            // e^{d h / eps}, d = 0 .. K / l + 1 grid steps
            const int nd = K / l + 2;
            hug.resize((size_t)nd * p->esz);
            for (int d = 0; d < nd; ++d) {
                const double e = std::exp((double)d * ugrid_h / eps);
                if (fp64)
                    reinterpret_cast<double *>(hug.data())[d] = e;
                else
                    reinterpret_cast<float *>(hug.data())[d] = (float)e;
            }
            ce = ce ? ce : up(p->ugrid, hug.data(), hug.size());
        } else {
            ce = ce ? ce : up(p->epos, hep.data(), hep.size());
            ce = ce ? ce : up(p->emid, hem.data(), hem.size());
        }
        ce = ce ? ce : up(p->ephi, hph.data(), hph.size());
        if (!fp64) {
            for (int k = 0; k < l && ce == cudaSuccess; ++k) {
                HVec<float2> ff(N[k]);
                const int64_t n = N[k];
                const std::vector<double> &lm = hlm[k];
                const int P = layout_threads(n);
                host_parallel(P, [&](int pp) {
                    for (int64_t i = n * pp / P; i < n * (pp + 1) / P; ++i) {
                        const double v = lm[i];
                        const float h = (float)v;
                        ff[i] = make_float2(h, std::isfinite(v) ? (float)(v - (double)h) : 0.0f);
                    }
                });
                ce = up(p->lnmu_ff[k], ff.data(), sizeof(float2) * N[k]);
                // the staging vector must outlive the copy
                if (ce == cudaSuccess) ce = cudaStreamSynchronize(p->st);
            }
        }
        // the staging vectors above go out of scope: wait for their copies
        ce = ce ? ce : cudaStreamSynchronize(p->st);
    }
    ce = ce ? ce : up(p->d_segt0, seg_tile0.data(), sizeof(int32_t) * (nin + 1));
    // carries of the empty state are never written by the level scans
    ce = ce ? ce : cudaMemsetAsync(p->fcarry, 0, (size_t)nt * p->NS * p->sfsz, p->st);
    ce = ce ? ce : cudaMemsetAsync(p->bcarry, 0, (size_t)nt * p->NS * p->sfsz, p->st);
    ce = ce ? ce : cudaMemsetAsync(p->err, 0, sizeof(int), p->st);
    ce = ce ? ce : cudaStreamSynchronize(p->st);
    if (ce != cudaSuccess) {
        delete p;
        return fail(MMOT_ERR_CUDA, "plan upload: %s", cudaGetErrorString(ce));
    }
    *out = p;
    return MMOT_OK;
}

// Objective terms of every instance of a plan (one for a single problem):
// residual over all l marginals, W, primal, dual and mass (Eq. k-mmot
// distance).  One product per marginal sums its terms per tile on the device
// (FP64), a compensated per-instance reduction follows, and the transport cost
// comes from the objective sweeps; only five FP64 values per instance reach
// the host.
// stop_res (optional): per instance the residual of the stopping test
// (marginals 1..l-1) from the same products
mmot_status plan_objective(mmot_plan p, std::vector<mmot_result> &R, std::vector<double> *stop_res = nullptr)
{
    const int l = p->l, ns = p->nseg;
    R.assign(ns, mmot_result{});
    CUDA_TRY(cudaMemsetAsync(p->d_obj, 0, sizeof(double) * 6 * ns, p->st));
    for (int k = 0; k < l; ++k) {
        mmot_status s = enqueue_product(p, k, MODE_OBJ, nullptr);
        if (s != MMOT_OK) return s;
        k_seg_obj<<<ns, 256, 0, p->st>>>(p->part4, nullptr, nullptr, p->d_segt0, p->d_obj, k == l - 1, k < l - 1);
        CUDA_TRY(cudaGetLastError());
        p->launches += 1;
    }
    const bool with_w = (l <= kMaxObjectiveL);
    if (with_w) {
        // transport cost: per instance, Z times the sum over its tiles of eps W_b / Z_b
        mmot_status sc = enqueue_cost(p);
        if (sc != MMOT_OK) return sc;
        k_seg_obj<<<ns, 256, 0, p->st>>>(nullptr, p->partial, p->o_lnz, p->d_segt0, p->d_obj, 0, 0);
        CUDA_TRY(cudaGetLastError());
        p->launches += 1;
    }
    std::vector<double> h((size_t)ns * 6);
    CUDA_TRY(cudaMemcpyAsync(h.data(), p->d_obj, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, p->st));
    CUDA_TRY(cudaStreamSynchronize(p->st));
    if (stop_res) stop_res->assign(ns, 0.0);
    for (int q = 0; q < ns; ++q) {
        const double e = p->seg_eps[q];
        const double *o = &h[(size_t)q * 6];
        if (stop_res) (*stop_res)[q] = o[5];
        R[q].mass = o[0];
        R[q].residual = o[1];
        R[q].primal = o[2];
        R[q].dual = o[3] + e - e * o[0];
        R[q].W = with_w ? o[4] : NAN;
    }
    return check_device_error(p);
}

}  // namespace

extern "C" {

const char *mmot_last_error(void) { return g_last_error.c_str(); }

void mmot_destroy(mmot_plan p)
{
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st);
    delete p;
}

mmot_status mmot_plan_create(int l, const int64_t *N, const double *const *x, const double *const *mu,
                             double eps, mmot_precision prec, int inputs_on_device, void *cuda_stream,
                             mmot_plan *out)
{
    g_last_error.clear();
    if (!out) return fail(MMOT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (l < 2 || l > MMOT_MAXL) return fail(MMOT_ERR_INVALID_ARG, "l = %d outside [2, 8]", l);
    if (!N || !x || !mu) return fail(MMOT_ERR_INVALID_ARG, "N, x or mu is NULL");
    std::vector<InstanceIn> ins(1);
    ins[0].N = N;
    ins[0].x = x;
    ins[0].mu = mu;
    ins[0].eps = eps;
    return plan_build(l, ins, prec, inputs_on_device, cuda_stream, out);
}

mmot_status mmot_marginal(mmot_plan p, int k, int plan_marginal, double *out)
{
    if (!p || !out) return fail(MMOT_ERR_INVALID_ARG, "NULL plan or out");
    if (k < 0 || k >= p->l) return fail(MMOT_ERR_INVALID_ARG, "marginal %d out of range", k);
    int mode;
    switch (plan_marginal) {
    case 0: mode = MODE_OUT_M; break;
    case 1: mode = MODE_OUT_PLAN; break;
    case 2: mode = MODE_OUT_LNM; break;
    default: return fail(MMOT_ERR_INVALID_ARG, "plan_marginal must be 0, 1 or 2");
    }
    const bool dev = is_device_ptr(out);
    double *dst = dev ? out : p->scratch;
    mmot_status s = enqueue_product(p, k, mode, dst);
    if (s != MMOT_OK) return s;
    if (!dev)
        CUDA_TRY(cudaMemcpyAsync(out, p->scratch, sizeof(double) * p->N[k], cudaMemcpyDeviceToHost, p->st));
    return check_device_error(p);
}

mmot_status mmot_sinkhorn_step(mmot_plan p, int n_iters, double *residual_out)
{
    if (!p) return fail(MMOT_ERR_INVALID_ARG, "NULL plan");
    if (p->shard) return fail(MMOT_ERR_INVALID_ARG, "shard plans iterate through mmot_shard_update");
    if (n_iters < 0) return fail(MMOT_ERR_INVALID_ARG, "n_iters < 0");
    if (n_iters > 0) {
        mmot_status s0 = ensure_ops(p, 0);
        if (s0 != MMOT_OK) return s0;
        if (p->use_graph && !p->profile) {
            if (!p->graph) {
                cudaGraph_t gr;
                CUDA_TRY(cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal));
                const int64_t before = p->launches;
                mmot_status s = enqueue_iteration(p);
                p->launches = before;   // captured, not launched
                cudaError_t e = cudaStreamEndCapture(p->st, &gr);
                if (s != MMOT_OK) return s;
                if (e != cudaSuccess) return fail(MMOT_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
                e = cudaGraphInstantiate(&p->graph, gr, 0);
                cudaGraphDestroy(gr);
                if (e != cudaSuccess) {
                    p->graph = nullptr;
                    return fail(MMOT_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
                }
            }
            for (int it = 0; it < n_iters; ++it) {
                CUDA_TRY(cudaGraphLaunch(p->graph, p->st));
                p->launches += (int64_t)p->l * launches_per_product(p);
            }
        } else {
            for (int it = 0; it < n_iters; ++it) {
                mmot_status s = enqueue_iteration(p);
                if (s != MMOT_OK) return s;
            }
        }
    }
    if (residual_out) {
        mmot_status s = enqueue_residual(p, 0, p->l - 1);
        if (s != MMOT_OK) return s;
        s = read_scalar(p, p->dsum, residual_out);
        if (s != MMOT_OK) return s;
    }
    return check_device_error(p);
}

mmot_status mmot_objective(mmot_plan p, mmot_result *out)
{
    if (!p || !out) return fail(MMOT_ERR_INVALID_ARG, "NULL plan or out");
    if (p->shard) return fail(MMOT_ERR_INVALID_ARG, "not on a shard plan");
    memset(out, 0, sizeof(*out));
    std::vector<mmot_result> R;
    mmot_status s = plan_objective(p, R);
    if (s != MMOT_OK) return s;
    *out = R[0];
    return MMOT_OK;
}

mmot_status mmot_solve(mmot_plan p, double tol, int itr_max, mmot_result *out)
{
    if (!p || !out) return fail(MMOT_ERR_INVALID_ARG, "NULL plan or out");
    if (p->shard) return fail(MMOT_ERR_INVALID_ARG, "shard plans iterate through mmot_shard_update");
    if (itr_max < 0) return fail(MMOT_ERR_INVALID_ARG, "itr_max < 0");
    int t = 0;
    double res = INFINITY;
    while (t < itr_max) {
        const int n = (tol > 0.0) ? std::min(p->check_every, itr_max - t) : itr_max - t;
        mmot_status s = mmot_sinkhorn_step(p, n, tol > 0.0 ? &res : nullptr);
        if (s != MMOT_OK) return s;
        t += n;
        if (tol > 0.0 && res <= tol) break;
    }
    // the objective's products give the stopping residual of the final
    // potentials as well (no separate residual products)
    memset(out, 0, sizeof(*out));
    std::vector<mmot_result> R;
    std::vector<double> stop;
    mmot_status s = plan_objective(p, R, &stop);
    if (s != MMOT_OK) return s;
    *out = R[0];
    if (tol <= 0.0 || t == 0) res = stop[0];
    out->iters = t;
    out->residual = res;
    s = check_device_error(p);
    if (s != MMOT_OK) return s;
    if (tol > 0.0 && res > tol) return fail(MMOT_ERR_NOT_CONVERGED, "residual %.3e > tol after %d iterations", res, t);
    return MMOT_OK;
}

mmot_status mmot_get_potentials(mmot_plan p, int k, double *g_out)
{
    if (!p || !g_out) return fail(MMOT_ERR_INVALID_ARG, "NULL plan or output");
    if (k < 0 || k >= p->l) return fail(MMOT_ERR_INVALID_ARG, "marginal %d out of range", k);
    CUDA_TRY(cudaMemcpyAsync(g_out, p->g[k], sizeof(double) * p->N[k], cudaMemcpyDefault, p->st));
    CUDA_TRY(cudaStreamSynchronize(p->st));
    return MMOT_OK;
}

mmot_status mmot_set_potentials(mmot_plan p, int k, const double *g_in)
{
    if (!p || !g_in) return fail(MMOT_ERR_INVALID_ARG, "NULL plan or input");
    if (k < 0 || k >= p->l) return fail(MMOT_ERR_INVALID_ARG, "marginal %d out of range", k);
    if (p->batch) {
        std::vector<double> g(p->N[k]);
        CUDA_TRY(cudaMemcpy(g.data(), g_in, sizeof(double) * p->N[k], cudaMemcpyDefault));
        for (int64_t i = 0; i < p->N[k]; ++i)
            if (std::isnan(g[i]) || g[i] == INFINITY)
                return fail(MMOT_ERR_INVALID_ARG, "g[%lld] is NaN or +inf", (long long)i);
        return upload_potential(p, k, g);
    }
    // on the device: the input into the plan's scratch (device input: after
    // all work queued on the device), a check for NaN / +inf (one flag read
    // back), then the copy into g_k and the re-centred stream copies
    const size_t nb = sizeof(double) * p->N[k];
    if (is_device_ptr(g_in)) {
        CUDA_TRY(cudaDeviceSynchronize());
        CUDA_TRY(cudaMemcpyAsync(p->scratch, g_in, nb, cudaMemcpyDeviceToDevice, p->st));
    } else {
        CUDA_TRY(cudaMemcpyAsync(p->scratch, g_in, nb, cudaMemcpyHostToDevice, p->st));
    }
    CUDA_TRY(cudaMemsetAsync(p->cflags, 0, sizeof(int), p->st));
    k_check_pot<<<64, 256, 0, p->st>>>(p->scratch, p->N[k], p->cflags);
    CUDA_TRY(cudaGetLastError());
    int bad = 0;
    CUDA_TRY(cudaMemcpyAsync(&bad, p->cflags, sizeof(int), cudaMemcpyDeviceToHost, p->st));
    CUDA_TRY(cudaStreamSynchronize(p->st));
    if (bad) return fail(MMOT_ERR_INVALID_ARG, "g contains NaN or +inf");
    CUDA_TRY(cudaMemcpyAsync(p->g[k], p->scratch, nb, cudaMemcpyDeviceToDevice, p->st));
    if (p->esz == 8)
        k_recentre<double><<<p->nt, 256, 0, p->st>>>(p->tstart, p->mid, p->cnt, p->toff, p->l, k, 1.0 / p->eps,
                                                     p->g[k], p->beta, static_cast<double *>(p->lphi),
                                                     p->three_phase ? static_cast<double *>(p->ephi) : nullptr);
    else
        k_recentre<float><<<p->nt, 256, 0, p->st>>>(p->tstart, p->mid, p->cnt, p->toff, p->l, k, 1.0 / p->eps,
                                                    p->g[k], p->beta, static_cast<float *>(p->lphi),
                                                    p->three_phase ? static_cast<float *>(p->ephi) : nullptr);
    CUDA_TRY(cudaGetLastError());
    p->launches += 3;
    CUDA_TRY(cudaStreamSynchronize(p->st));
    p->ops_target = -1;
    return MMOT_OK;
}

mmot_status mmot_set_option(mmot_plan p, int option, int64_t value)
{
    if (!p) return fail(MMOT_ERR_INVALID_ARG, "NULL plan");
    switch (option) {
    case MMOT_OPT_CHECK_EVERY:
        if (value < 1) return fail(MMOT_ERR_INVALID_ARG, "check_every must be >= 1");
        p->check_every = (int)value;
        return MMOT_OK;
    case MMOT_OPT_SPIN_LIMIT:
        if (value < 1 || value > (1LL << 30)) return fail(MMOT_ERR_INVALID_ARG, "spin limit out of range");
        p->spin_limit = (int)value;
        if (p->graph) {
            cudaGraphExecDestroy(p->graph);
            p->graph = nullptr;
        }
        return MMOT_OK;
    case MMOT_OPT_USE_GRAPH:
        p->use_graph = value ? 1 : 0;
        return MMOT_OK;
    case MMOT_OPT_PROFILE:
        p->profile = value ? 1 : 0;
        return MMOT_OK;
    case MMOT_OPT_TEST_HOLD:
        p->hold = value ? 1 : 0;
        if (p->graph) {
            cudaGraphExecDestroy(p->graph);
            p->graph = nullptr;
        }
        return MMOT_OK;
    default: return fail(MMOT_ERR_INVALID_ARG, "unknown option %d", option);
    }
}

mmot_status mmot_reset_potentials(mmot_plan p)
{
    if (!p) return fail(MMOT_ERR_INVALID_ARG, "NULL plan");
    const int l = p->l;
    for (int k = 0; k < l; ++k) {
        if (p->batch)
            k_reset_seg<<<p->nseg, 256, 0, p->st>>>(p->g[k], p->d_goff, p->d_g0, k, l);
        else
            k_reset<<<64, 256, 0, p->st>>>(p->g[k], p->N[k], -p->eps * std::log((double)p->Ninit[k]));
        CUDA_TRY(cudaGetLastError());
        p->launches += 1;
    }
    if (p->batch) CUDA_TRY(cudaMemsetAsync(p->d_frozen, 0, sizeof(int32_t) * p->nseg, p->st));
    p->h_beta = p->h_beta0;
    CUDA_TRY(cudaMemcpyAsync(p->beta, p->h_beta.data(), sizeof(double) * p->h_beta.size(),
                             cudaMemcpyHostToDevice, p->st));
    CUDA_TRY(cudaMemsetAsync(p->lphi, 0, (size_t)p->T * p->esz, p->st));
    if (p->three_phase) {
        if (p->esz == 8)
            k_fill<double><<<256, 256, 0, p->st>>>(static_cast<double *>(p->ephi), p->Tpad, 1.0);
        else
            k_fill<float><<<256, 256, 0, p->st>>>(static_cast<float *>(p->ephi), p->Tpad, 1.0f);
        CUDA_TRY(cudaGetLastError());
        p->launches += 1;
    }
    p->ops_target = -1;
    return MMOT_OK;
}

mmot_status mmot_get_profile(mmot_plan p, int kernel, int64_t *launches, double *total_ms, int reset)
{
    if (!p || !launches || !total_ms) return fail(MMOT_ERR_INVALID_ARG, "NULL argument");
    if (kernel < 0 || kernel > 7) return fail(MMOT_ERR_INVALID_ARG, "kernel must be in 0..7");
    CUDA_TRY(cudaStreamSynchronize(p->st));
    for (auto &r : p->recs) {
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
        p->prof_count[r.kernel] += 1;
        p->prof_ms[r.kernel] += ms;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    p->recs.clear();
    *launches = p->prof_count[kernel];
    *total_ms = p->prof_ms[kernel];
    if (reset) {
        for (int q = 0; q < 7; ++q) {
            p->prof_count[q] = 0;
            p->prof_ms[q] = 0.0;
        }
    }
    return MMOT_OK;
}

mmot_status mmot_get_info(mmot_plan p, mmot_plan_info *info)
{
    if (!p || !info) return fail(MMOT_ERR_INVALID_ARG, "NULL plan or info");
    info->total_points = p->T;
    info->tiles = p->nt;
    info->tile_points = p->K;
    info->threads_per_block = p->NT;
    info->launches_per_iteration = p->l * launches_per_product(p);
    info->precision = p->prec;
    info->kernel_launches = p->launches;
    info->device_bytes = p->dev_bytes;
    info->uniform_grid = (p->ugrid != nullptr) ? 1 : 0;
    return MMOT_OK;
}

mmot_status mmot_set_memory_limit(int64_t bytes)
{
    if (bytes < 0) return fail(MMOT_ERR_INVALID_ARG, "memory limit < 0");
    g_mem_limit = bytes;
    return MMOT_OK;
}

mmot_status mmot_memory_in_use(int64_t *bytes)
{
    if (!bytes) return fail(MMOT_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = g_mem_used.load();
    return MMOT_OK;
}

// ---- shards of one instance ----------------------------------------------------

mmot_status mmot_shard_create(int l, const int64_t *N, const double *const *x, const double *const *mu,
                              const int64_t *N_total, double eps, mmot_precision prec, int inputs_on_device,
                              void *cuda_stream, mmot_plan *out)
{
    g_last_error.clear();
    if (!out) return fail(MMOT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (l < 2 || l > MMOT_MAXL) return fail(MMOT_ERR_INVALID_ARG, "l = %d outside [2, 8]", l);
    if (!N || !x || !mu || !N_total) return fail(MMOT_ERR_INVALID_ARG, "N, x, mu or N_total is NULL");
    if (l - 1 > kMaxOpBits) return fail(MMOT_ERR_RANGE, "shards need l <= %d (tile operators), got l = %d", kMaxOpBits + 1, l);
    for (int k = 0; k < l; ++k)
        if (N_total[k] < N[k])
            return fail(MMOT_ERR_INVALID_ARG, "N_total[%d] = %lld < N[%d] = %lld", k, (long long)N_total[k], k,
                        (long long)N[k]);
    std::vector<InstanceIn> ins(1);
    ins[0].N = N;
    ins[0].x = x;
    ins[0].mu = mu;
    ins[0].eps = eps;
    ins[0].Ntot = N_total;
    return plan_build(l, ins, prec, inputs_on_device, cuda_stream, out);
}

mmot_status mmot_shard_operator(mmot_plan p, int k, double *lnop)
{
    if (!p || !lnop) return fail(MMOT_ERR_INVALID_ARG, "NULL plan or lnop");
    if (!p->shard) return fail(MMOT_ERR_INVALID_ARG, "not a shard plan");
    if (k < 0 || k >= p->l) return fail(MMOT_ERR_INVALID_ARG, "marginal %d out of range", k);
    mmot_status s = ensure_ops(p, k);
    if (s != MMOT_OK) return s;
    SweepArgs a = make_args(p, k, MODE_UPDATE, nullptr);
    CUDA_TRY(launch_opc(p->NB, a, p->prec == MMOT_FP64, p->st, p->d_lnop));
    p->launches += 1;
    const size_t n = (size_t)2 * (p->NB + 1) * p->NS;
    CUDA_TRY(cudaMemcpyAsync(lnop, p->d_lnop, sizeof(double) * n, cudaMemcpyDefault, p->st));
    return check_device_error(p);
}

mmot_status mmot_shard_set_inflow(mmot_plan p, int k, const double *lnF, const double *lnG)
{
    if (!p) return fail(MMOT_ERR_INVALID_ARG, "NULL plan");
    if (!p->shard) return fail(MMOT_ERR_INVALID_ARG, "not a shard plan");
    if (k < 0 || k >= p->l) return fail(MMOT_ERR_INVALID_ARG, "marginal %d out of range", k);
    const int NS = p->NS;
    const bool fp64 = (p->prec == MMOT_FP64);
    std::vector<unsigned char> h((size_t)2 * NS * p->sfsz, 0);
    for (int d = 0; d < 2; ++d) {
        const double *src = d ? lnG : lnF;
        for (int T = 1; T < NS; ++T) {
            const double y = src ? src[T] : -INFINITY;
            if (std::isnan(y) || y == INFINITY)
                return fail(MMOT_ERR_INVALID_ARG, "inflow %s[%d] is not finite or -inf", d ? "lnG" : "lnF", T);
            if (y == -INFINITY) continue;
            // m 2^e with m in [0.5, 1): e = floor(y / ln 2) + 1
            const double t = y / std::log(2.0);
            const double n = std::floor(t);
            int e = 0;
            const double m = std::frexp(std::exp2(t - n), &e);
            const long long kk = (long long)n + e;
            if (fp64) {
                double *q = reinterpret_cast<double *>(h.data()) + 2 * ((size_t)d * NS + T);
                q[0] = m;
                q[1] = (double)kk;
            } else {
                float *q = reinterpret_cast<float *>(h.data()) + 2 * ((size_t)d * NS + T);
                const int ki = (int)kk;
                q[0] = (float)m;
                std::memcpy(&q[1], &ki, sizeof(int));
            }
        }
    }
    CUDA_TRY(cudaMemcpyAsync(p->inflow, h.data(), h.size(), cudaMemcpyHostToDevice, p->st));
    CUDA_TRY(cudaStreamSynchronize(p->st));
    p->inflow_target = k;
    return MMOT_OK;
}

mmot_status mmot_shard_update(mmot_plan p, int k)
{
    if (!p) return fail(MMOT_ERR_INVALID_ARG, "NULL plan");
    if (!p->shard) return fail(MMOT_ERR_INVALID_ARG, "not a shard plan");
    if (k < 0 || k >= p->l) return fail(MMOT_ERR_INVALID_ARG, "marginal %d out of range", k);
    if (p->inflow_target != k) return fail(MMOT_ERR_INVALID_ARG, "no inflow set for marginal %d", k);
    mmot_status s = enqueue_product(p, k, MODE_UPDATE, nullptr, (k + 1) % p->l);
    if (s != MMOT_OK) return s;
    return check_device_error(p);
}

mmot_status mmot_shard_residual(mmot_plan p, int k, double *res)
{
    if (!p || !res) return fail(MMOT_ERR_INVALID_ARG, "NULL plan or res");
    if (!p->shard) return fail(MMOT_ERR_INVALID_ARG, "not a shard plan");
    if (k < 0 || k >= p->l) return fail(MMOT_ERR_INVALID_ARG, "marginal %d out of range", k);
    if (p->inflow_target != k) return fail(MMOT_ERR_INVALID_ARG, "no inflow set for marginal %d", k);
    mmot_status s = enqueue_residual(p, k, k + 1);
    if (s != MMOT_OK) return s;
    s = read_scalar(p, p->dsum, res);
    if (s != MMOT_OK) return s;
    return check_device_error(p);
}

// ---- batches ------------------------------------------------------------------

}  // extern "C"

struct mmot_batch_s {
    int n = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    struct Group {
        int l = 0;
        mmot_plan p = nullptr;
        std::vector<int> inst;        // batch index of each instance of the group
        std::vector<int> iters;       // iterations when found converged (else run so far)
        std::vector<double> res;      // last checked residual
        std::vector<int32_t> conv;    // converged (frozen)
        std::vector<int32_t> frozen_only;   // frozen by the caller without converging
        int done = 0;                 // iterations run on the group
        int active = 0;
    };
    std::vector<Group> groups;
    std::vector<std::pair<int, int>> where;   // instance -> (group, index in group)
    ~mmot_batch_s()
    {
        for (auto &g : groups) mmot_destroy(g.p);
        if (own_stream && st) cudaStreamDestroy(st);
    }
};

namespace {

// per-instance residual of marginals 1..l-1 of a group; freeze the converged
mmot_status group_check(mmot_batch_s::Group &G, double tol)
{
    mmot_plan p = G.p;
    const int ns = p->nseg;
    CUDA_TRY(cudaMemsetAsync(p->d_res, 0, sizeof(double) * ns, p->st));
    for (int k = 0; k < p->l - 1; ++k) {
        mmot_status s = enqueue_product(p, k, MODE_RESIDUAL, nullptr);
        if (s != MMOT_OK) return s;
        k_seg_sum<<<(ns + 127) / 128, 128, 0, p->st>>>(p->partial, p->d_segt0, ns, p->d_res, 1);
        CUDA_TRY(cudaGetLastError());
        p->launches += 1;
    }
    std::vector<double> r(ns);
    CUDA_TRY(cudaMemcpyAsync(r.data(), p->d_res, sizeof(double) * ns, cudaMemcpyDeviceToHost, p->st));
    CUDA_TRY(cudaStreamSynchronize(p->st));
    int active = 0;
    bool changed = false;
    for (int q = 0; q < ns; ++q) {
        if (G.conv[q] || G.frozen_only[q]) continue;
        G.res[q] = r[q];
        G.iters[q] = G.done;
        if (r[q] <= tol) {
            G.conv[q] = 1;
            changed = true;
        } else {
            ++active;
        }
    }
    G.active = active;
    if (changed) {
        std::vector<int32_t> fz(ns);
        for (int q = 0; q < ns; ++q) fz[q] = G.conv[q] | G.frozen_only[q];
        CUDA_TRY(cudaMemcpyAsync(p->d_frozen, fz.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, p->st));
        CUDA_TRY(cudaStreamSynchronize(p->st));
    }
    return check_device_error(p);
}

mmot_status group_reset(mmot_batch_s::Group &G)
{
    mmot_status s = mmot_reset_potentials(G.p);
    if (s != MMOT_OK) return s;
    const int ns = (int)G.inst.size();
    G.iters.assign(ns, 0);
    G.res.assign(ns, INFINITY);
    G.conv.assign(ns, 0);
    G.frozen_only.assign(ns, 0);
    G.done = 0;
    G.active = ns;
    return MMOT_OK;
}

}  // namespace

extern "C" {

mmot_status mmot_batch_create(int n, const int *l, const int64_t *N, const double *const *x,
                              const double *const *mu, const double *eps, mmot_precision prec,
                              int tile_points, void *cuda_stream, mmot_batch *out)
{
    g_last_error.clear();
    if (!out) return fail(MMOT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !l || !N || !x || !mu || !eps) return fail(MMOT_ERR_INVALID_ARG, "n < 1 or NULL argument");
    if (tile_points < 0) return fail(MMOT_ERR_INVALID_ARG, "tile_points < 0");
    std::vector<int64_t> off(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        if (l[i] < 2 || l[i] > MMOT_MAXL) return fail(MMOT_ERR_INVALID_ARG, "instance %d: l = %d outside [2, 8]", i, l[i]);
        off[i + 1] = off[i] + l[i];
    }
    mmot_batch b = new (std::nothrow) mmot_batch_s();
    if (!b) return fail(MMOT_ERR_OOM, "host allocation failed");
    b->n = n;
    if (cuda_stream) {
        b->st = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return fail(MMOT_ERR_CUDA, "stream creation failed: %s", cudaGetErrorString(e));
        }
        b->own_stream = true;
    }
    b->where.assign(n, {-1, -1});
    for (int L = 2; L <= MMOT_MAXL; ++L) {
        std::vector<InstanceIn> ins;
        std::vector<int> idx;
        for (int i = 0; i < n; ++i) {
            if (l[i] != L) continue;
            InstanceIn in;
            in.N = N + off[i];
            in.x = x + off[i];
            in.mu = mu + off[i];
            in.eps = eps[i];
            ins.push_back(in);
            idx.push_back(i);
        }
        if (ins.empty()) continue;
        // one group per l; a group with more tiles than one carry scan takes
        // is split into consecutive parts
        std::vector<std::pair<size_t, size_t>> todo{{0, ins.size()}};
        while (!todo.empty()) {
            const auto r = todo.back();
            todo.pop_back();
            std::vector<InstanceIn> part(ins.begin() + r.first, ins.begin() + r.second);
            mmot_batch_s::Group G;
            G.l = L;
            mmot_status s = plan_build(L, part, prec, 0, b->st, &G.p, tile_points, true);
            if (s == MMOT_ERR_RANGE && r.second - r.first > 1) {
                const size_t mid = (r.first + r.second) / 2;
                todo.push_back({mid, r.second});
                todo.push_back({r.first, mid});
                continue;
            }
            if (s != MMOT_OK) {
                std::string m = g_last_error;
                delete b;
                return fail(s, "l = %d group: %s", L, m.c_str());
            }
            G.inst.assign(idx.begin() + r.first, idx.begin() + r.second);
            for (size_t q = 0; q < G.inst.size(); ++q) b->where[G.inst[q]] = {(int)b->groups.size(), (int)q};
            b->groups.push_back(G);
            s = group_reset(b->groups.back());
            if (s != MMOT_OK) {
                delete b;
                return s;
            }
        }
    }
    *out = b;
    return MMOT_OK;
}

mmot_status mmot_batch_reset(mmot_batch b)
{
    if (!b) return fail(MMOT_ERR_INVALID_ARG, "NULL batch");
    for (auto &G : b->groups) {
        mmot_status s = group_reset(G);
        if (s != MMOT_OK) return s;
    }
    return MMOT_OK;
}

mmot_status mmot_batch_step(mmot_batch b, int n_iters, double tol, int *active_out)
{
    if (!b) return fail(MMOT_ERR_INVALID_ARG, "NULL batch");
    if (n_iters < 0) return fail(MMOT_ERR_INVALID_ARG, "n_iters < 0");
    int active = 0;
    for (auto &G : b->groups) {
        if (G.active == 0) continue;
        mmot_status s = mmot_sinkhorn_step(G.p, n_iters, nullptr);
        if (s != MMOT_OK) return s;
        G.done += n_iters;
        s = group_check(G, tol);
        if (s != MMOT_OK) return s;
        active += G.active;
    }
    if (active_out) *active_out = active;
    return MMOT_OK;
}

mmot_status mmot_batch_solve(mmot_batch b, double tol, int itr_max, int check_every, mmot_result *results)
{
    if (!b) return fail(MMOT_ERR_INVALID_ARG, "NULL batch");
    if (itr_max < 0 || check_every < 1) return fail(MMOT_ERR_INVALID_ARG, "itr_max < 0 or check_every < 1");
    mmot_status s = mmot_batch_reset(b);
    if (s != MMOT_OK) return s;
    int t = 0, active = b->n;
    while (t < itr_max && active > 0) {
        const int n = std::min(check_every, itr_max - t);
        s = mmot_batch_step(b, n, tol, &active);
        if (s != MMOT_OK) return s;
        t += n;
    }
    if (itr_max == 0) {
        for (auto &G : b->groups) {
            s = group_check(G, tol);
            if (s != MMOT_OK) return s;
        }
    }
    if (results) {
        for (auto &G : b->groups) {
            std::vector<mmot_result> R;
            s = plan_objective(G.p, R);
            if (s != MMOT_OK) return s;
            for (size_t q = 0; q < G.inst.size(); ++q) {
                mmot_result r = R[q];
                r.iters = G.iters[q];
                r.residual = G.res[q];
                results[G.inst[q]] = r;
            }
        }
    }
    for (auto &G : b->groups)
        if (G.active > 0) return fail(MMOT_ERR_NOT_CONVERGED, "%d instance(s) with l = %d above tol after %d iterations",
                                      G.active, G.l, t);
    return MMOT_OK;
}

mmot_status mmot_batch_freeze(mmot_batch b, int i)
{
    if (!b) return fail(MMOT_ERR_INVALID_ARG, "NULL batch");
    if (i < 0 || i >= b->n) return fail(MMOT_ERR_INVALID_ARG, "instance %d out of range", i);
    auto &G = b->groups[b->where[i].first];
    const int q = b->where[i].second;
    if (G.frozen_only[q] || G.conv[q]) return MMOT_OK;
    G.frozen_only[q] = 1;
    G.active -= 1;
    const int32_t one = 1;
    CUDA_TRY(cudaMemcpyAsync(G.p->d_frozen + q, &one, sizeof(int32_t), cudaMemcpyHostToDevice, G.p->st));
    CUDA_TRY(cudaStreamSynchronize(G.p->st));
    return MMOT_OK;
}

mmot_status mmot_batch_status(mmot_batch b, int i, int *iters, double *residual, int *converged)
{
    if (!b) return fail(MMOT_ERR_INVALID_ARG, "NULL batch");
    if (i < 0 || i >= b->n) return fail(MMOT_ERR_INVALID_ARG, "instance %d out of range", i);
    const auto &G = b->groups[b->where[i].first];
    const int q = b->where[i].second;
    if (iters) *iters = G.iters[q];
    if (residual) *residual = G.res[q];
    if (converged) *converged = G.conv[q];
    return MMOT_OK;
}

mmot_status mmot_batch_get_potentials(mmot_batch b, int i, int k, double *g_out)
{
    if (!b || !g_out) return fail(MMOT_ERR_INVALID_ARG, "NULL batch or output");
    if (i < 0 || i >= b->n) return fail(MMOT_ERR_INVALID_ARG, "instance %d out of range", i);
    const auto &G = b->groups[b->where[i].first];
    const int q = b->where[i].second;
    mmot_plan p = G.p;
    if (k < 0 || k >= p->l) return fail(MMOT_ERR_INVALID_ARG, "marginal %d out of range", k);
    const int64_t o = p->seg_off[(size_t)q * p->l + k];
    const int64_t n = p->seg_off[(size_t)(q + 1) * p->l + k] - o;
    CUDA_TRY(cudaMemcpyAsync(g_out, p->g[k] + o, sizeof(double) * n, cudaMemcpyDefault, p->st));
    CUDA_TRY(cudaStreamSynchronize(p->st));
    return MMOT_OK;
}

mmot_status mmot_batch_set_potentials(mmot_batch b, int i, int k, const double *g_in)
{
    if (!b || !g_in) return fail(MMOT_ERR_INVALID_ARG, "NULL batch or input");
    if (i < 0 || i >= b->n) return fail(MMOT_ERR_INVALID_ARG, "instance %d out of range", i);
    auto &G = b->groups[b->where[i].first];
    const int q = b->where[i].second;
    mmot_plan p = G.p;
    if (k < 0 || k >= p->l) return fail(MMOT_ERR_INVALID_ARG, "marginal %d out of range", k);
    const int64_t o = p->seg_off[(size_t)q * p->l + k];
    const int64_t n = p->seg_off[(size_t)(q + 1) * p->l + k] - o;
    std::vector<double> gi((size_t)n);
    if (is_device_ptr(g_in)) CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpyAsync(gi.data(), g_in, sizeof(double) * n, cudaMemcpyDefault, p->st));
    CUDA_TRY(cudaStreamSynchronize(p->st));
    for (int64_t t = 0; t < n; ++t)
        if (std::isnan(gi[t]) || gi[t] == INFINITY)
            return fail(MMOT_ERR_INVALID_ARG, "g[%lld] is NaN or +inf", (long long)t);
    // the group's marginal k with this instance's slice replaced, then the
    // host re-centring of the whole marginal (ln phi and e^{ln phi} streams)
    std::vector<double> g((size_t)p->N[k]);
    CUDA_TRY(cudaMemcpyAsync(g.data(), p->g[k], sizeof(double) * p->N[k], cudaMemcpyDeviceToHost, p->st));
    CUDA_TRY(cudaStreamSynchronize(p->st));
    std::copy(gi.begin(), gi.end(), g.begin() + o);
    mmot_status s = upload_potential(p, k, g);
    if (s != MMOT_OK) return s;
    if (G.conv[q] || G.frozen_only[q]) {
        G.conv[q] = 0;
        G.frozen_only[q] = 0;
        G.active += 1;
        const int32_t zero = 0;
        CUDA_TRY(cudaMemcpyAsync(p->d_frozen + q, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, p->st));
        CUDA_TRY(cudaStreamSynchronize(p->st));
    }
    G.res[q] = NAN;
    return MMOT_OK;
}

mmot_status mmot_batch_get_info(mmot_batch b, mmot_batch_info *info)
{
    if (!b || !info) return fail(MMOT_ERR_INVALID_ARG, "NULL batch or info");
    info->instances = b->n;
    info->groups = (int)b->groups.size();
    info->total_points = 0;
    info->tiles = 0;
    info->kernel_launches = 0;
    for (auto &G : b->groups) {
        info->total_points += G.p->T;
        info->tiles += G.p->nt;
        info->kernel_launches += G.p->launches;
    }
    return MMOT_OK;
}

void mmot_batch_destroy(mmot_batch b)
{
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    delete b;
}

}  // extern "C"
