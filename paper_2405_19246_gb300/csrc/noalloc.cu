// mmot_marginal_noalloc: one marginal product without any device allocation.
//
// Some callers cannot allocate device memory: code that runs under a memory
// manager with a fixed device budget (a framework's caching pool that owns all
// device memory), plug-ins that must not change the process's allocation
// state, or latency-critical loops where cudaMalloc's implicit device
// synchronisation is not acceptable.  They bring their own input and output
// buffers; everything else this call needs lives in the file-scope array
// below, which every GPU that loads the library holds until the process
// exits.
//
// The computation is the same as mmot_marginal on a plan (FP32 in-tile scans,
// three-phase tile operators / carry scan / tile products): merge, tiling and
// the padded exponential stream on the host, tables copied into the static
// scratch, three kernel launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/mmot.h"
#include "layout.h"
#include "mmot_internal.cuh"
#include "shapes.cuh"

namespace {

using namespace mmot;

constexpr size_t kScratchBytes = size_t(8) << 20;   // 8 MiB per device
constexpr int64_t kMaxPoints = int64_t(1) << 19;     // sum_k N_k
constexpr int kMaxTiles = 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// device address of g_scratch, looked up once per device with that device current
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

template <int NB>
void shape_f32(int *K, int *jcap)
{
    *K = TShape<NB, float>::K;
    *jcap = TShape<NB, float>::JCAP;
}

mmot_status err_msg(mmot_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return set_error(st, buf);
}

#define NA_TRY(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return err_msg(MMOT_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));           \
    } while (0)

}  // namespace

extern "C" mmot_status mmot_marginal_noalloc(int l, const int64_t *N, const double *const *x,
                                             const double *const *g, double eps, int k, int plan_marginal,
                                             double *out, void *cuda_stream)
{
    set_error(MMOT_OK, "");
    if (l < 2 || l > kMaxOpBits + 1)
        return err_msg(MMOT_ERR_RANGE, "mmot_marginal_noalloc supports 2 <= l <= %d, got l = %d", kMaxOpBits + 1, l);
    if (!N || !x || !g || !out) return err_msg(MMOT_ERR_INVALID_ARG, "NULL argument");
    if (!(eps > 0.0) || !std::isfinite(eps)) return err_msg(MMOT_ERR_INVALID_ARG, "eps must be positive and finite");
    if (k < 0 || k >= l) return err_msg(MMOT_ERR_INVALID_ARG, "marginal %d out of range", k);
    int mode;
    switch (plan_marginal) {
    case 0: mode = MODE_OUT_M; break;
    case 1: mode = MODE_OUT_PLAN; break;
    case 2: mode = MODE_OUT_LNM; break;
    default: return err_msg(MMOT_ERR_INVALID_ARG, "plan_marginal must be 0, 1 or 2");
    }
    int64_t T = 0;
    for (int q = 0; q < l; ++q) {
        if (N[q] < 1) return err_msg(MMOT_ERR_INVALID_ARG, "N[%d] = %lld < 1", q, (long long)N[q]);
        if (!x[q] || !g[q]) return err_msg(MMOT_ERR_INVALID_ARG, "x[%d] or g[%d] is NULL", q, q);
        T += N[q];
    }
    if (T > kMaxPoints)
        return err_msg(MMOT_ERR_RANGE, "mmot_marginal_noalloc: sum N = %lld exceeds the static scratch limit of %lld points",
                       (long long)T, (long long)kMaxPoints);
    auto on_device = [](const void *ptr) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return at.type == cudaMemoryTypeDevice;
    };
    if (!on_device(out)) return err_msg(MMOT_ERR_INVALID_ARG, "out must be device memory");
    if (mode == MODE_OUT_PLAN && !on_device(g[k]))
        return err_msg(MMOT_ERR_INVALID_ARG, "g[k] must be device memory for plan_marginal = 1");
    int dev = 0;
    NA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return err_msg(MMOT_ERR_RANGE, "device index %d too large", dev);
    unsigned char *scratch;
    {
        // first call on this device: look up the address of the static array
        // (a host-side name is not a device address)
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            NA_TRY(cudaGetSymbolAddress(&ptr, g_scratch));
            g_scratch_addr[dev] = static_cast<unsigned char *>(ptr);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // ---- inputs to the host (cudaMemcpyDefault: host or device pointers) ----
    // The reads are issued on the caller's stream, so they are ordered after
    // whatever the caller queued there (for example the kernel that wrote g).
    std::vector<std::vector<double>> hx(l), hg(l);
    for (int q = 0; q < l; ++q) {
        hx[q].resize(N[q]);
        hg[q].resize(N[q]);
        NA_TRY(cudaMemcpyAsync(hx[q].data(), x[q], sizeof(double) * N[q], cudaMemcpyDefault, st));
        NA_TRY(cudaMemcpyAsync(hg[q].data(), g[q], sizeof(double) * N[q], cudaMemcpyDefault, st));
    }
    NA_TRY(cudaStreamSynchronize(st));
    for (int q = 0; q < l; ++q) {
        for (int64_t i = 0; i < N[q]; ++i) {
            if (!std::isfinite(hx[q][i])) return err_msg(MMOT_ERR_INVALID_ARG, "x[%d][%lld] not finite", q, (long long)i);
            if (i > 0 && hx[q][i] < hx[q][i - 1])
                return err_msg(MMOT_ERR_UNSORTED, "x[%d] decreases at index %lld", q, (long long)i);
            if (std::isnan(hg[q][i]) || hg[q][i] == INFINITY)
                return err_msg(MMOT_ERR_INVALID_ARG, "g[%d][%lld] is NaN or +inf", q, (long long)i);
        }
    }

    // ---- layout --------------------------------------------------------------
    const int NB = l - 1;
    const int NS = 1 << NB;
    int K = 0, jcap = 0;
    switch (NB) {
    case 1: shape_f32<1>(&K, &jcap); break;
    case 2: shape_f32<2>(&K, &jcap); break;
    case 3: shape_f32<3>(&K, &jcap); break;
    default: shape_f32<4>(&K, &jcap); break;
    }
    HostLayout L;
    build_layout(l, N, hx, eps, K, jcap, kSpanLimitF32, L);
    const int nt = L.nt;
    if (nt > kMaxTiles)
        return err_msg(MMOT_ERR_RANGE, "mmot_marginal_noalloc: %d tiles exceed the static scratch limit of %d", nt, kMaxTiles);
    // baselines: the per-tile maximum of g_m/eps (0 when none is finite);
    // ln phi is stored relative to them
    std::vector<double> beta((size_t)nt * l, 0.0);
    std::fill(beta.begin(), beta.end(), -INFINITY);
    for (int q = 0; q < l; ++q)
        for (int64_t i = 0; i < N[q]; ++i) {
            const uint32_t t = L.mpos[q][i];
            double &bq = beta[(size_t)L.tile_of[t] * l + q];
            bq = std::max(bq, hg[q][i] / eps);
        }
    for (double &bq : beta)
        if (!std::isfinite(bq)) bq = 0.0;
    // padded stream of the tile kernels: every tile starts on a 16-element
    // boundary; e^{pos}, scaled phi e^{g/eps - beta}, marginal (0xff: padding)
    std::vector<uint32_t> htoff(nt);
    int64_t Tp = 0;
    for (int b = 0; b < nt; ++b) {
        htoff[b] = (uint32_t)Tp;
        Tp += ((int64_t)(L.tstart[b + 1] - L.tstart[b]) + 15) / 16 * 16;
    }
    std::vector<float> hepos(Tp, 1.0f), hephi(Tp, 0.0f);
    std::vector<uint8_t> hemid(Tp, 0xff);
    for (int b = 0; b < nt; ++b)
        for (uint32_t t = L.tstart[b]; t < L.tstart[b + 1]; ++t) {
            const size_t u = (size_t)htoff[b] + (t - L.tstart[b]);
            hepos[u] = (float)std::exp(L.pos[t]);
            hemid[u] = L.mid[t];
        }
    for (int q = 0; q < l; ++q)
        for (int64_t i = 0; i < N[q]; ++i) {
            const uint32_t t = L.mpos[q][i];
            const uint32_t b = L.tile_of[t];
            hephi[(size_t)htoff[b] + (t - L.tstart[b])] = (float)std::exp(hg[q][i] / eps - beta[(size_t)b * l + q]);
        }
    std::vector<unsigned char> decF, decB;
    decay_tables(L, NB, false, decF, decB);

    // ---- scratch layout ------------------------------------------------------
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_epos = take(sizeof(float) * Tp);
    const size_t o_ephi = take(sizeof(float) * Tp);
    const size_t o_emid = take((size_t)Tp);
    const size_t o_toff = take(sizeof(uint32_t) * nt);
    const size_t o_ts = take(sizeof(uint32_t) * (nt + 1));
    const size_t o_ulb = take(sizeof(double) * nt);
    const size_t o_urb = take(sizeof(double) * nt);
    const size_t o_span = take(sizeof(double) * nt);
    const size_t o_cnt = take(sizeof(int32_t) * nt * l);
    const size_t o_ref = take(sizeof(int32_t) * nt * l);
    const size_t o_beta = take(sizeof(double) * nt * l);
    const size_t o_decF = take(decF.size());
    const size_t o_decB = take(decB.size());
    const size_t o_opF = take(sizeof(float2) * nt * NB * NS);
    const size_t o_opB = take(sizeof(float2) * nt * NB * NS);
    const size_t o_fc = take(sizeof(float2) * nt * NS);
    const size_t o_bc = take(sizeof(float2) * nt * NS);
    const size_t o_cfl = take(sizeof(int) * 2 * 32 * l);
    const size_t o_cag = take(sizeof(float2) * 2 * 32 * NS);
    const size_t o_err = take(sizeof(int));
    if (off > kScratchBytes) return err_msg(MMOT_ERR_RANGE, "problem needs %zu scratch bytes > %zu", off, kScratchBytes);
    std::vector<unsigned char> stage(o_opF, 0);   // everything the host fills
    auto put = [&](size_t o, const void *src, size_t bytes) { std::memcpy(stage.data() + o, src, bytes); };
    put(o_epos, hepos.data(), sizeof(float) * Tp);
    put(o_ephi, hephi.data(), sizeof(float) * Tp);
    put(o_emid, hemid.data(), (size_t)Tp);
    put(o_toff, htoff.data(), sizeof(uint32_t) * nt);
    put(o_ts, L.tstart.data(), sizeof(uint32_t) * (nt + 1));
    put(o_ulb, L.ulb.data(), sizeof(double) * nt);
    put(o_urb, L.urb.data(), sizeof(double) * nt);
    put(o_span, L.span.data(), sizeof(double) * nt);
    put(o_cnt, L.cnt.data(), sizeof(int32_t) * nt * l);
    put(o_ref, L.reftile.data(), sizeof(int32_t) * nt * l);
    put(o_beta, beta.data(), sizeof(double) * nt * l);
    put(o_decF, decF.data(), decF.size());
    put(o_decB, decB.data(), decB.size());
    NA_TRY(cudaMemcpyAsync(scratch, stage.data(), stage.size(), cudaMemcpyHostToDevice, st));
    // the error word must start at zero on every call (the array keeps the
    // previous call's contents)
    NA_TRY(cudaMemsetAsync(scratch + o_err, 0, sizeof(int), st));
    // the carry-scan flags must start at zero too
    NA_TRY(cudaMemsetAsync(scratch + o_cfl, 0, sizeof(int) * 2 * 32 * l, st));

    // ---- kernels ---------------------------------------------------------------
    SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.l = l;
    a.j = k;
    a.nt = nt;
    a.mode = mode;
    a.eps = eps;
    a.inv_eps = 1.0 / eps;
    a.tstart = reinterpret_cast<const uint32_t *>(scratch + o_ts);
    a.ulb = reinterpret_cast<const double *>(scratch + o_ulb);
    a.urb = reinterpret_cast<const double *>(scratch + o_urb);
    a.span = reinterpret_cast<const double *>(scratch + o_span);
    a.cnt = reinterpret_cast<const int32_t *>(scratch + o_cnt);
    a.reftile = reinterpret_cast<const int32_t *>(scratch + o_ref);
    a.beta = reinterpret_cast<double *>(scratch + o_beta);
    a.epos = scratch + o_epos;
    a.ephi = scratch + o_ephi;
    a.emid = scratch + o_emid;
    a.toff = reinterpret_cast<const uint32_t *>(scratch + o_toff);
    a.opF = scratch + o_opF;
    a.opB = scratch + o_opB;
    a.fcarry = scratch + o_fc;
    a.bcarry = scratch + o_bc;
    a.pdecF = scratch + o_decF;
    a.pdecB = scratch + o_decB;
    a.gj = const_cast<double *>(g[k]);
    a.out = out;
    a.err = reinterpret_cast<int *>(scratch + o_err);
    a.cflags = reinterpret_cast<int *>(scratch + o_cfl);
    a.cagg = scratch + o_cag;
    a.spin_limit = 1 << 23;
    a.jnext = -1;
    for (int kind = 2; kind <= 4; ++kind) NA_TRY(launch_three_phase(NB, a, false, st, kind));
    int herr = 0;
    NA_TRY(cudaMemcpyAsync(&herr, scratch + o_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
    if (herr & ERR_TIMEOUT) return err_msg(MMOT_ERR_TIMEOUT, "an inter-tile wait reached its poll limit");
    if (herr & ERR_RANGE) return err_msg(MMOT_ERR_RANGE, "a tile exceeded its target-point capacity");
    if (herr & ERR_NONFINITE) return err_msg(MMOT_ERR_NONFINITE, "a product became NaN or infinite");
    if (herr) return err_msg(MMOT_ERR_CUDA, "kernel error flags %d", herr);
    return MMOT_OK;
}
