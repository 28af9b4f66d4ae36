// Host checks of the merged-order tiling (layout.h): tie order, tile limits,
// per-marginal counts, and the batch layout (instances one after another,
// no decay across an instance boundary).  Prints "ok" or the first failure.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <tuple>
#include <vector>

#include "layout.h"

using namespace mmot;

#define CHECK(c)                                                         \
    do {                                                                 \
        if (!(c)) {                                                      \
            std::printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c);      \
            std::exit(1);                                                \
        }                                                                \
    } while (0)

static double dec_value(const std::vector<unsigned char> &T, size_t idx)
{
    const float *q = reinterpret_cast<const float *>(T.data()) + 2 * idx;
    int k;
    std::memcpy(&k, &q[1], sizeof(int));
    return q[0] == 0.f ? 0.0 : std::ldexp((double)q[0], k);
}

int main()
{
    // three marginals with shared coordinates: ties go to the lower marginal
    const int l = 3;
    std::vector<std::vector<double>> x = {{0.0, 0.5, 0.5, 1.0}, {0.5, 0.7}, {0.1, 0.5, 0.9}};
    int64_t N[3] = {4, 2, 3};
    HostLayout L;
    build_layout(l, N, x, 0.1, 4, 2, 24.0, L);
    CHECK(L.T == 9);
    // merged order by (x, marginal, index)
    for (int64_t t = 1; t < L.T; ++t) {
        CHECK(L.xm[t - 1] <= L.xm[t]);
        if (L.xm[t - 1] == L.xm[t]) CHECK(L.mid[t - 1] <= L.mid[t]);
    }
    // every local point maps to its merged position
    for (int k = 0; k < l; ++k)
        for (int64_t i = 0; i < N[k]; ++i) {
            const uint32_t t = L.mpos[k][i];
            CHECK(L.mid[t] == k && L.xm[t] == x[k][i]);
        }
    // tiles: at most K points, at most jcap of one marginal, span limit, counts
    for (int b = 0; b < L.nt; ++b) {
        const int n = (int)(L.tstart[b + 1] - L.tstart[b]);
        CHECK(n >= 1 && n <= 4);
        int per[3] = {0, 0, 0};
        for (uint32_t t = L.tstart[b]; t < L.tstart[b + 1]; ++t) per[L.mid[t]]++;
        for (int k = 0; k < l; ++k) CHECK(per[k] <= 2);
        CHECK(L.span[b] * 2.0 <= 24.0 + 1e-12);
        for (int k = 0; k < l; ++k) {
            int before = 0;
            for (uint32_t t = 0; t < L.tstart[b]; ++t) before += (L.mid[t] == k);
            CHECK(L.cnt[(size_t)b * l + k] == before);
        }
    }

    // batch: two instances appended; counts move by the first instance's sizes
    std::vector<std::vector<double>> y = {{0.2, 0.4}, {0.3}, {0.25, 0.6}};
    int64_t M[3] = {2, 1, 2};
    HostLayout Ly;
    build_layout(l, M, y, 0.05, 4, 2, 24.0, Ly);
    HostLayout B;
    B.l = l;
    std::vector<int64_t> off(l, 0);
    append_layout(B, L, off.data());
    for (int k = 0; k < l; ++k) off[k] = N[k];
    append_layout(B, Ly, off.data());
    CHECK(B.T == L.T + Ly.T && B.nt == L.nt + Ly.nt);
    // appending to an empty layout gives the layout itself (plan creation
    // takes a single instance's layout as it is)
    {
        HostLayout E;
        E.l = l;
        std::vector<int64_t> zero(l, 0);
        append_layout(E, L, zero.data());
        CHECK(E.T == L.T && E.nt == L.nt && E.tstart == L.tstart && E.cnt == L.cnt && E.reftile == L.reftile);
        CHECK(E.mid == L.mid && E.pos == L.pos && E.tile_of == L.tile_of && E.span == L.span);
        CHECK(E.xlb == L.xlb && E.xrb == L.xrb && E.ulb == L.ulb && E.urb == L.urb);
        for (int k = 0; k < l; ++k) CHECK(E.mpos[k] == L.mpos[k]);
    }
    CHECK(B.tstart.size() == (size_t)B.nt + 1 && B.tstart.back() == (uint32_t)B.T);
    std::vector<int32_t> seg;
    for (int b = 0; b < L.nt; ++b) seg.push_back(0);
    for (int b = 0; b < Ly.nt; ++b) seg.push_back(1);
    for (int b = 0; b < Ly.nt; ++b)
        for (int k = 0; k < l; ++k) {
            const int bb = L.nt + b;
            CHECK(B.cnt[(size_t)bb * l + k] == Ly.cnt[(size_t)b * l + k] + (int32_t)N[k]);
            CHECK(B.reftile[(size_t)bb * l + k] >= L.nt);   // stays inside its instance
        }
    for (int k = 0; k < l; ++k)
        for (int64_t i = 0; i < M[k]; ++i) CHECK(B.mpos[k][N[k] + i] == Ly.mpos[k][i] + (uint32_t)L.T);
    // decays: exp(-w_s d) inside an instance, 0 across the boundary and out of the last tile
    std::vector<unsigned char> F, Bk;
    decay_tables(B, l - 1, false, F, Bk, seg);
    const int NB1 = l;
    for (int b = 0; b < B.nt; ++b)
        for (int s = 1; s < NB1; ++s) {
            const double w = (double)s * (l - s);
            const double f = dec_value(F, (size_t)b * NB1 + s);
            if (b + 1 < B.nt && seg[b + 1] == seg[b]) {
                const double ref = std::exp(-w * (B.ulb[b + 1] - B.ulb[b]));
                CHECK(std::fabs(f - ref) <= 1e-6 * ref);
            } else {
                CHECK(f == 0.0);
            }
            const double g = dec_value(Bk, (size_t)b * NB1 + s);
            if (b >= 1 && seg[b - 1] == seg[b]) {
                const double ref = std::exp(-w * (B.urb[b] - B.urb[b - 1]));
                CHECK(std::fabs(g - ref) <= 1e-6 * ref);
            } else {
                CHECK(g == 0.0);
            }
        }

    // above a million points the merge and the per-tile pass run on host
    // threads in parts: the merged order must still be the sort by
    // (x, marginal, index), with ties (a coarse grid of values) across parts
    {
        const int lb = 4;
        std::mt19937_64 rng(5);
        std::vector<std::vector<double>> z(lb);
        int64_t Nz[4];
        std::vector<std::tuple<double, int, int64_t>> ref;
        for (int k = 0; k < lb; ++k) {
            Nz[k] = 280000 + (int64_t)(rng() % 20000);
            z[k].resize(Nz[k]);
            for (auto &v : z[k]) v = (double)(rng() % 50000) / 50000.0;
            std::sort(z[k].begin(), z[k].end());
            for (int64_t i = 0; i < Nz[k]; ++i) ref.emplace_back(z[k][i], k, i);
        }
        std::sort(ref.begin(), ref.end());
        HostLayout Z;
        build_layout(lb, Nz, z, 1e-3, 2048, 544, 24.0, Z);
        CHECK(Z.T == (int64_t)ref.size() && Z.T >= (1 << 20));
        for (int64_t t = 0; t < Z.T; ++t) {
            CHECK(Z.xm[t] == std::get<0>(ref[t]) && Z.mid[t] == std::get<1>(ref[t]));
            CHECK(Z.mpos[std::get<1>(ref[t])][std::get<2>(ref[t])] == (uint32_t)t);
        }
        int64_t covered = 0;
        for (int b = 0; b < Z.nt; ++b)
            for (uint32_t t = Z.tstart[b]; t < Z.tstart[b + 1]; ++t) {
                CHECK(Z.tile_of[t] == (uint32_t)b);
                CHECK(Z.pos[t] == (Z.xm[t] - Z.xlb[b]) / 1e-3);
                ++covered;
            }
        CHECK(covered == Z.T);

        // padded stream: tile b's points at toff[b] + (t - tstart[b]); e^{pos},
        // ephi 1 and the marginal there, and 1 / 0 / 0xff in the padding
        std::vector<uint32_t> toff(Z.nt);
        int64_t o = 0;
        for (int b = 0; b < Z.nt; ++b) {
            toff[b] = (uint32_t)o;
            o += ((int64_t)(Z.tstart[b + 1] - Z.tstart[b]) + 15) / 16 * 16;
        }
        const size_t Tp = (size_t)o;
        HVec<float> ep(Tp), ph(Tp);
        HVec<uint8_t> em(Tp);
        fill_padded_stream<float>(Z.nt, Z.tstart.data(), toff.data(), Tp, Z.pos.data(), Z.mid.data(), ep.data(),
                                  ph.data(), em.data());
        std::vector<char> seen(Tp, 0);
        for (int b = 0; b < Z.nt; ++b)
            for (uint32_t t = Z.tstart[b]; t < Z.tstart[b + 1]; ++t) {
                const size_t u = toff[b] + (t - Z.tstart[b]);
                CHECK(ep[u] == (float)std::exp(Z.pos[t]) && ph[u] == 1.0f && em[u] == Z.mid[t]);
                seen[u] = 1;
            }
        for (size_t u = 0; u < Tp; ++u)
            if (!seen[u]) CHECK(ep[u] == 1.0f && ph[u] == 0.0f && em[u] == 0xff);
        HVec<float> pc(Z.T);
        convert_parallel(Z.T, Z.pos.data(), pc.data());
        for (int64_t t = 0; t < Z.T; ++t) CHECK(pc[t] == (float)Z.pos[t]);
    }
    std::printf("ok\n");
    return 0;
}
