// Internal declarations shared by the host runtime and the sweep kernels.
//
// Terminology (arXiv 2405.19246, Sec. 3 and Sec. 4.2):
//   merged order  all sum_k N_k support points sorted by (x, marginal, index);
//                 the tie rule of the order classes D_p (Eq. D_p).
//   target j      the marginal whose product M_j is evaluated; the other
//                 marginals R = [l] \ {j} are mapped to bits 0..l-2.
//   state S       a subset of R; F_S(z) sums over placements of one point of
//                 each marginal of S left of z of prod phi * exp(-cost so far),
//                 G_S(z) is the mirror image right of z.  Orderings that put
//                 the same set left of z share one state: these are the
//                 paper's class chains (Sec. 4.2) with shared prefixes.
//   rate w_s      s(l-s): while s tuple points lie left of z, s(l-s) pairs
//                 straddle z, so every state with |S| = s decays as
//                 exp(-s(l-s) dx / eps) (the multiplier lambda^2 of
//                 Algorithm 2 is the l = 3 case, w_1 = w_2 = 2).
//   M_j(i)        sum_S F_S(x_i^-) G_{R\S}(x_i^+)   (Eq. Jk k margin).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define MMOT_MAXL 8

namespace mmot {

enum Mode : int {
    MODE_UPDATE = 0,       // g_j <- eps (ln mu_j - ln M_j), refresh ln phi_j copy
    MODE_OUT_M = 1,        // out[i] = M_j(i)
    MODE_OUT_PLAN = 2,     // out[i] = phi_j(i) M_j(i)
    MODE_OUT_LNM = 3,      // out[i] = ln M_j(i)
    MODE_RESIDUAL = 4,     // partial[b] = sum over tile of |phi_j M_j - mu_j|
    MODE_OBJ = 5,          // part4[b] = tile sums of marg_j, |marg_j - mu_j|, g_j marg_j, g_j mu_j
};

enum ErrBits : int {
    ERR_TIMEOUT = 1,
    ERR_NONFINITE = 2,
    ERR_RANGE = 4,
};

// Everything a sweep kernel reads or writes; passed by value.
struct SweepArgs {
    int l;           // marginals
    int j;           // target marginal
    int nt;          // tiles
    int mode;
    int spin_limit;  // polls before a wait gives up
    int hold;        // test hook: the first chunk of a carry scan never publishes its flags
    double eps;
    double inv_eps;
    // per tile
    const uint32_t *tstart;   // [nt+1] first merged index of each tile
    const double *ulb;        // [nt]   x/eps of the first point of the tile
    const double *urb;        // [nt]   x/eps of the last point of the tile
    const double *span;       // [nt]   (xrb - xlb)/eps
    const int32_t *cnt;       // [nt*l] points of marginal m before tile b
    const int32_t *reftile;   // [nt*l] tile whose beta represents marginal m in tile b
    double *beta;             // [nt*l] per-tile baseline of g_m/eps
    // the same points in the padded stream of the tile kernels (l <= 5):
    // tile b occupies [toff[b], toff[b] + n_b), toff[b] a multiple of 16;
    // FP32 or FP64 values
    const uint32_t *toff;     // [nt] stream offset of each tile
    const void *epos;         // e^{(x_t - x_first_of_tile)/eps}
    void *ephi;               // e^{g_m(i)/eps - beta[b*l+m]}
    const uint8_t *emid;      // marginal of the point, 0xff for padding
    const float2 *lnmuj_ff;   // [N_j] ln mu_j as FP32 hi + lo (FP32 path)
    // per merged point
    // FP32 arrays for the FP32 path, FP64 arrays for the all-FP64 path
    const void *pos;          // (x_t - xlb[b])/eps
    const uint8_t *mid;       // marginal of the point
    void *lphi;               // g_m(i)/eps - beta[b*l+m]
    // inter-tile scan state, indexed by processing order v
    // values are scaled floats (m, k) = m * 2^k, stored as float2 (FP32 path,
    // k in the bits of .y) or double2 (FP64 path)
    void *agg;                // [nt*NS] the tile's own contribution at its base
    void *inc;                // [nt*NS] inclusive prefix at the tile's base
    int *flags;               // [nt*(NB+1)] 0 none, 1 aggregate, 2 inclusive, 3 failed
    int *counter;             // dynamic tile counter
    void *bcarry;             // [nt*NS] backward carries at each tile's right end
    void *fcarry;             // [nt*NS] forward carries at each tile's left end
    // carry-free tile transfer operators (decay to the next tile base
    // included): op[(b*NB + s)*NS + U], forward and backward
    void *opF;
    void *opB;
    // exp(-w_s d) from each tile base to the next one in processing order,
    // [nt*(NB+1)], forward and backward
    const void *pdecF;
    const void *pdecB;
    int jnext;                // target of the operators computed after an update (-1: none)
    // level passes of l >= 6 taking two levels per walk: the pass of level s
    // also leaves level s+1's contributions that do not go through a level-s
    // carry, and per tile and marginal the coefficient with which a level-s
    // carry reaches level s+1 (coef, [nt*NB] scaled floats); the scan of
    // level s+1 adds the carries' share (pair = 1 in both launches)
    void *coef;
    int pair;
    // shards of one instance (shard.cuh): the states entering the range
    // ([dir][NS] scaled floats, absolute, at the left end forward and the right
    // end backward; null: only the empty state), and whether the last tile in
    // processing order carries its operator and decay to the range's end
    const void *inflow;
    int shard_end;
    // tile kernels (l <= 5): every lane's chunk transfer operators of the
    // current target, [tile][dir][entry][lane] (null: recomputed by a walk)
    void *lops;
    // all marginals on one uniform grid (x_i = x_0 + i h): merged point t is
    // grid point t / l of marginal t % l, and ugrid[d] = e^{d h / eps} (V) for
    // d grid steps from the tile's first point; epos and emid are not read
    // (null: the general stream)
    const void *ugrid;
    // warp tiles (l >= 6): backward states at the target points of the
    // current target marginal, [target point][2^(l-1)] scaled floats
    void *gtarg;
    // carry scan over chunks of tiles: flags [2][G][NB+1], contributions [2][G][NS]
    int *cflags;
    void *cagg;
    // target marginal
    double *gj;               // [N_j] potentials (FP64)
    const double *lnmuj;      // [N_j] ln mu_j (-inf for zero weights)
    const double *muj;        // [N_j] mu_j
    double *out;              // [N_j] output for the OUT modes
    double *partial;          // [nt] per-tile residual sums
    double *part4;            // [nt*4] per-tile objective sums (MODE_OBJ)
    int *err;                 // error bits
    // batches of independent instances (all NULL for a single instance):
    // tiles never straddle two instances and no state crosses a boundary
    const int32_t *seg;       // [nt] instance of each tile (nondecreasing)
    const double *teps;       // [nt] eps of each tile's instance
    const int32_t *frozen;    // [instances] nonzero: updates and residual terms skipped
};

// eps of tile b
__host__ __device__ inline double tile_eps(const SweepArgs &a, int b) { return a.teps ? a.teps[b] : a.eps; }

// Host-side launchers (one per bit count NB = l-1, instantiated per precision).
// Three-phase design (l <= 5): tile operators, carry scan over tiles, tile
// products with known carries (optionally followed by the operators of a.jnext).
template <int NB, typename V>
cudaError_t launch_tileop(const SweepArgs &a, cudaStream_t s);
template <int NB, typename V>
cudaError_t launch_carry(const SweepArgs &a, cudaStream_t s);
template <int NB, typename V>
cudaError_t launch_prod(const SweepArgs &a, cudaStream_t s);
// Level passes (l >= 6): tile contributions of one level, scalar carry scan.
template <int NB, typename V>
cudaError_t launch_lagg(const SweepArgs &a, cudaStream_t s, int level, int fwd);
template <int NB, typename V>
cudaError_t launch_lscan(const SweepArgs &a, cudaStream_t s, int level, int fwd);
// Backward walk of the warp-tile products (l >= 6): states at the targets.
template <int NB, typename V>
cudaError_t launch_wbwd(const SweepArgs &a, cudaStream_t s);
// Transfer operator of a whole shard from the tile operators (shard.cuh):
// lnop[2][NB + 1][2^NB] natural logarithms, device memory.
template <int NB, typename V>
cudaError_t launch_opcompose(const SweepArgs &a, cudaStream_t s, double *lnop);
constexpr int kMaxOpBits = 4;
// message for mmot_last_error (defined in mmot.cu)
}  // namespace mmot
#include "../../include/mmot.h"
namespace mmot {
mmot_status set_error(mmot_status st, const char *msg);
// kind: 2 tile operators, 3 carry scan, 4 tile products (defined in mmot.cu)
cudaError_t launch_three_phase(int NB, const SweepArgs &a, bool fp64, cudaStream_t st, int kind);

// Objective sweeps of l marginals (l state bits, no target; objective.cuh).
// kind: 0 backward look-back sweep (l >= 5), 2 tile operators, 3 carry scan
// (l <= 4), 5 objective kernel.
template <int L, typename V>
cudaError_t launch_objective(const SweepArgs &a, cudaStream_t s, int kind);
// Objective sweeps of l = 8 marginals on warp tiles (warp.cuh): kind 5 level
// pass, 6 level scan, 7 objective kernel.
template <typename V>
cudaError_t launch_objective_warp8(const SweepArgs &a, cudaStream_t s, int kind, int level, int fwd);
constexpr int kMaxObjectiveL = 8;

// Tile geometry chosen per (bits, precision): points per tile, threads,
// maximum points of one marginal in a tile, and the tile span limit
// max_s w_s * span (keeps in-tile exponents small).
struct TileShape {
    int K;
    int NT;
    int JCAP;
    double span_limit;
};
TileShape tile_shape(int NB, bool fp64);

}  // namespace mmot
