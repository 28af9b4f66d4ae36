// Host-side layout of one problem: the merged order of all support points
// and its tiling (shared by mmot_plan_create and mmot_marginal_noalloc).
//
// Merged order: all T = sum_k N_k points sorted by (x, marginal, index); ties
// between marginals go to the lower marginal index first, the tie rule of the
// order classes D_p (Eq. D_p).
// Tiles: consecutive runs of the merged order with at most K points, at most
// jcap points of any one marginal, and max_s w_s * (x_last - x_first)/eps at
// most `limit` (w_s = s(l - s)).
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <thread>
#include <type_traits>
#include <utility>
#include <vector>

#include "mmot_internal.cuh"

namespace mmot {

// Allocator whose resize leaves new elements of a trivial type uninitialised:
// the per-point layout arrays are written once, in parallel, by the threads
// that own their parts, so a value-initialising resize would only zero them
// serially first (and take every page fault on one thread).
template <typename T>
struct DefaultInit : std::allocator<T> {
    using std::allocator<T>::allocator;
    DefaultInit() = default;
    template <typename U>
    DefaultInit(const DefaultInit<U> &) noexcept {}
    template <typename U>
    struct rebind {
        using other = DefaultInit<U>;
    };
    template <typename U>
    void construct(U *p) noexcept(std::is_nothrow_default_constructible<U>::value)
    {
        ::new (static_cast<void *>(p)) U;
    }
    template <typename U, typename... A>
    void construct(U *p, A &&...a)
    {
        ::new (static_cast<void *>(p)) U(std::forward<A>(a)...);
    }
};
template <typename T>
using HVec = std::vector<T, DefaultInit<T>>;

struct HostLayout {
    int l = 0;
    int64_t T = 0;
    int nt = 0;
    HVec<double> xm;                         // merged coordinates
    HVec<uint8_t> mid;                       // marginal of each merged point
    HVec<uint32_t> mpos[MMOT_MAXL];          // merged index of each local point
    std::vector<uint32_t> tstart;            // [nt+1]
    HVec<uint32_t> tile_of;                  // tile of each merged point
    std::vector<double> xlb, xrb;            // first / last x of each tile
    std::vector<double> ulb, urb, span;      // the same divided by eps; span = urb - ulb
    HVec<double> pos;                        // (x_t - xlb[tile])/eps
    std::vector<int32_t> cnt;                // [nt*l] points of marginal m before tile b
    std::vector<int32_t> reftile;            // [nt*l] nearest tile holding points of m
};

// f(part) for part = 0..parts-1 on up to `parts` host threads
template <typename F>
inline void host_parallel(int parts, F &&f)
{
    if (parts <= 1) {
        f(0);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(parts - 1);
    for (int p = 1; p < parts; ++p) th.emplace_back([&f, p] { f(p); });
    f(0);
    for (auto &t : th) t.join();
}

// host threads for a layout of T points (one below a million points)
inline int layout_threads(int64_t T)
{
    if (T < (1 << 20)) return 1;
    const unsigned hc = std::thread::hardware_concurrency();
    return (int)std::min<unsigned>(16u, std::max(1u, hc));
}

// hx[k]: the sorted coordinates of marginal k (any random-access container)
template <typename XS>
inline void build_layout(int l, const int64_t *N, const XS &hx, double eps, int K, int jcap, double limit,
                         HostLayout &L)
{
    L.l = l;
    int64_t T = 0;
    for (int k = 0; k < l; ++k) T += N[k];
    L.T = T;
    L.xm.resize(T);
    L.mid.resize(T);
    for (int k = 0; k < l; ++k) L.mpos[k].resize(N[k]);
    {
        // The merge in P independent parts: part p takes, of every marginal,
        // the points with x in [v_p, v_{p+1}) (split values from the largest
        // marginal), so equal coordinates never straddle two parts and each
        // part's merged offset is the number of points below v_p.
        const int P = layout_threads(T);
        int kbig = 0;
        for (int k = 1; k < l; ++k)
            if (N[k] > N[kbig]) kbig = k;
        std::vector<std::vector<int64_t>> lo(P + 1, std::vector<int64_t>(l, 0));
        for (int k = 0; k < l; ++k) lo[P][k] = N[k];
        for (int p = 1; p < P; ++p) {
            const double v = hx[kbig][(size_t)(N[kbig] * p / P)];
            for (int k = 0; k < l; ++k)
                lo[p][k] = std::lower_bound(hx[k].begin(), hx[k].end(), v) - hx[k].begin();
        }
        host_parallel(P, [&](int p) {
            std::vector<int64_t> head(lo[p]);
            int64_t t = 0;
            for (int k = 0; k < l; ++k) t += lo[p][k];
            int64_t tend = 0;
            for (int k = 0; k < l; ++k) tend += lo[p + 1][k];
            for (; t < tend; ++t) {
                int best = -1;
                for (int k = 0; k < l; ++k) {
                    if (head[k] >= lo[p + 1][k]) continue;
                    if (best < 0 || hx[k][head[k]] < hx[best][head[best]]) best = k;
                }
                L.xm[t] = hx[best][head[best]];
                L.mid[t] = (uint8_t)best;
                L.mpos[best][head[best]] = (uint32_t)t;
                head[best] += 1;
            }
        });
    }
    double wmax = 0.0;
    for (int s = 0; s <= l; ++s) wmax = std::max(wmax, (double)s * (l - s));
    L.tstart.clear();
    {
        int64_t t = 0;
        std::vector<int> per(l, 0);
        while (t < T) {
            L.tstart.push_back((uint32_t)t);
            const double x0 = L.xm[t];
            std::fill(per.begin(), per.end(), 0);
            per[L.mid[t]] = 1;
            int64_t e = t + 1;
            while (e < T && e - t < K && (L.xm[e] - x0) / eps * wmax <= limit && per[L.mid[e]] < jcap) {
                per[L.mid[e]] += 1;
                ++e;
            }
            t = e;
        }
        L.tstart.push_back((uint32_t)T);
    }
    const int nt = (int)L.tstart.size() - 1;
    L.nt = nt;
    L.tile_of.resize(T);
    L.xlb.resize(nt);
    L.xrb.resize(nt);
    L.ulb.resize(nt);
    L.urb.resize(nt);
    L.span.resize(nt);
    L.pos.resize(T);
    L.cnt.assign((size_t)nt * l, 0);
    L.reftile.assign((size_t)nt * l, -1);
    {
        // per tile (in parallel): ends, positions, tile of each point and the
        // tile's points per marginal; then the counts before each tile
        const int P = layout_threads(T);
        host_parallel(P, [&](int p) {
            for (int b = (int)((int64_t)nt * p / P); b < (int)((int64_t)nt * (p + 1) / P); ++b) {
                L.xlb[b] = L.xm[L.tstart[b]];
                L.xrb[b] = L.xm[L.tstart[b + 1] - 1];
                L.ulb[b] = L.xlb[b] / eps;
                L.urb[b] = L.xrb[b] / eps;
                L.span[b] = (L.xrb[b] - L.xlb[b]) / eps;
                for (uint32_t t = L.tstart[b]; t < L.tstart[b + 1]; ++t) {
                    L.pos[t] = (L.xm[t] - L.xlb[b]) / eps;
                    L.tile_of[t] = (uint32_t)b;
                    L.cnt[(size_t)b * l + L.mid[t]] += 1;
                    L.reftile[(size_t)b * l + L.mid[t]] = b;
                }
            }
        });
        std::vector<int32_t> run(l, 0);
        for (int b = 0; b < nt; ++b)
            for (int k = 0; k < l; ++k) {
                const int32_t c = L.cnt[(size_t)b * l + k];
                L.cnt[(size_t)b * l + k] = run[k];
                run[k] += c;
            }
    }
    // tiles without points of marginal m use the nearest earlier tile that has
    // some, else the nearest later one
    for (int k = 0; k < l; ++k) {
        int last = -1;
        for (int b = 0; b < nt; ++b) {
            int32_t &r = L.reftile[(size_t)b * l + k];
            if (r == b) last = b;
            else r = last;
        }
        int next = -1;
        for (int b = nt - 1; b >= 0; --b) {
            int32_t &r = L.reftile[(size_t)b * l + k];
            if (r == b) next = b;
            else if (r < 0) r = next;
        }
    }
}

// Append the layout of one more instance (batches): merged indices, tiles and
// the per-marginal counts move by the sizes already present; marg_off[k] is
// the number of points of marginal k before the instance.
inline void append_layout(HostLayout &D, const HostLayout &S, const int64_t *marg_off)
{
    const uint32_t toff = (uint32_t)D.T;
    const int32_t boff = D.nt;
    const int l = S.l;
    D.l = l;
    D.mid.insert(D.mid.end(), S.mid.begin(), S.mid.end());
    D.pos.insert(D.pos.end(), S.pos.begin(), S.pos.end());
    for (int k = 0; k < l; ++k)
        for (uint32_t t : S.mpos[k]) D.mpos[k].push_back(t + toff);
    if (!D.tstart.empty()) D.tstart.pop_back();
    for (uint32_t t : S.tstart) D.tstart.push_back(t + toff);
    for (uint32_t b : S.tile_of) D.tile_of.push_back(b + (uint32_t)boff);
    D.xlb.insert(D.xlb.end(), S.xlb.begin(), S.xlb.end());
    D.xrb.insert(D.xrb.end(), S.xrb.begin(), S.xrb.end());
    D.ulb.insert(D.ulb.end(), S.ulb.begin(), S.ulb.end());
    D.urb.insert(D.urb.end(), S.urb.begin(), S.urb.end());
    D.span.insert(D.span.end(), S.span.begin(), S.span.end());
    for (int b = 0; b < S.nt; ++b)
        for (int k = 0; k < l; ++k) {
            D.cnt.push_back(S.cnt[(size_t)b * l + k] + (int32_t)marg_off[k]);
            D.reftile.push_back(S.reftile[(size_t)b * l + k] + boff);
        }
    D.T += S.T;
    D.nt += S.nt;
}

// The padded stream of the tile kernels (l <= 5): tile b's points at
// toff[b] + (t - tstart[b]), each tile starting on a 16-element boundary and
// the last one padded to Tp.  epos = e^{pos} (skipped when null: uniform
// grids form it on the device), ephi = e^{ln phi} of ln phi = 0 (1 at a point,
// 0 in the padding), emid = the point's marginal (0xff in the padding).  Every
// element is written once, by the host thread that owns its tile.
template <typename Tv>
inline void fill_padded_stream(int nt, const uint32_t *tstart, const uint32_t *toff, size_t Tp, const double *pos,
                               const uint8_t *mid, Tv *epos, Tv *ephi, uint8_t *emid)
{
    const int P = layout_threads((int64_t)Tp);
    host_parallel(P, [&](int pp) {
        for (int b = (int)((int64_t)nt * pp / P); b < (int)((int64_t)nt * (pp + 1) / P); ++b) {
            const size_t u0 = toff[b], u1 = (b + 1 < nt) ? (size_t)toff[b + 1] : Tp;
            const size_t n = tstart[b + 1] - tstart[b];
            for (size_t i = 0; i < n; ++i) {
                const size_t u = u0 + i, t = tstart[b] + i;
                ephi[u] = Tv(1);
                if (epos) {
                    epos[u] = (Tv)std::exp(pos[t]);
                    emid[u] = mid[t];
                }
            }
            for (size_t u = u0 + n; u < u1; ++u) {
                ephi[u] = Tv(0);
                if (epos) {
                    epos[u] = Tv(1);
                    emid[u] = 0xff;
                }
            }
        }
    });
}

// values converted to the stream precision, on host threads
template <typename Tv>
inline void convert_parallel(int64_t n, const double *src, Tv *dst)
{
    const int P = layout_threads(n);
    host_parallel(P, [&](int pp) {
        for (int64_t i = n * pp / P; i < n * (pp + 1) / P; ++i) dst[i] = (Tv)src[i];
    });
}

// exp(-w_s d) from each tile base to the next base in processing order
// (forward: left ends, backward: right ends), s = 0..NB, as scaled floats
// m * 2^k stored as float2 (k in the bits of .y) or double2.  The decay out
// of the last tile, and across the boundary between two instances of a batch
// (seg, one entry per tile, may be empty), is 0: no state crosses it.  With
// to_end (shards of one instance) the last tile in processing order decays
// to the range's own end instead (forward x_R, backward x_L).
inline void decay_tables(const HostLayout &L, int NB, bool fp64, std::vector<unsigned char> &F,
                         std::vector<unsigned char> &B, const std::vector<int32_t> &seg = {}, bool to_end = false)
{
    const int nt = L.nt;
    const int l = L.l;
    const int NB1 = NB + 1;
    const size_t sz = fp64 ? 16 : 8;
    F.assign((size_t)nt * NB1 * sz, 0);
    B.assign((size_t)nt * NB1 * sz, 0);
    auto put = [&](std::vector<unsigned char> &dst, size_t idx, double lnv) {
        const double y = lnv / std::log(2.0);
        const bool zero = !(y >= -1.0e9);
        const double n = zero ? 0.0 : std::floor(y);
        int e = 0;
        const double m = std::frexp(std::exp2(zero ? 0.0 : y - n), &e);
        const long long k = (long long)n + e;
        if (fp64) {
            double *q = reinterpret_cast<double *>(dst.data()) + 2 * idx;
            q[0] = zero ? 0.0 : m;
            q[1] = zero ? 0.0 : (double)k;
        } else {
            float *q = reinterpret_cast<float *>(dst.data()) + 2 * idx;
            const int ki = zero ? 0 : (int)k;
            q[0] = zero ? 0.0f : (float)m;
            std::memcpy(&q[1], &ki, sizeof(int));
        }
    };
    auto same = [&](int b0, int b1) { return seg.empty() || seg[b0] == seg[b1]; };
    for (int b = 0; b < nt; ++b) {
        const bool okF = (b + 1 < nt) && same(b, b + 1);
        const bool okB = (b >= 1) && same(b - 1, b);
        const bool endF = to_end && b + 1 == nt, endB = to_end && b == 0;
        const double dF = okF ? L.ulb[b + 1] - L.ulb[b] : (endF ? L.span[b] : 0.0);
        const double dB = okB ? L.urb[b] - L.urb[b - 1] : (endB ? L.span[b] : 0.0);
        for (int s = 0; s < NB1; ++s) {
            const double ws = (double)s * (double)(l - s);
            put(F, (size_t)b * NB1 + s, (okF || endF) ? -ws * dF : -INFINITY);
            put(B, (size_t)b * NB1 + s, (okB || endB) ? -ws * dB : -INFINITY);
        }
    }
}

}  // namespace mmot
