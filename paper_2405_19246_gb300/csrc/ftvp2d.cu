// Fast tensor-vector product of the two-dimensional problem (Sec. 4.1, "High
// dimension generalization"; Algorithm 6, FTVP_2d): three marginals on one
// uniform N x M grid, L1 cost with steps h1 (first index) and h2 (second), so
// the kernel is separable, K = K1 (x) K2 with
//     Kd(i, j, k) = lam_d^{|i-j| + |i-k| + |j-k|} = mu_d^{max(i,j,k) - min(i,j,k)},
// mu_d = lam_d^2, and the product
//     J(k1, k2) = sum_{i1,i2,j1,j2} K1(i1,j1,k1) K2(i2,j2,k2) phi(i1,i2) psi(j1,j2).
//
// One dimension at a time.  In one dimension, for target index k,
//     sum_{i,j} mu^{max - min} a_i b_j = X_ab(k) + mu Y_ab(k+1)
//                                        + mu X_a(k) Y_b(k+1) + mu X_b(k) Y_a(k+1)
// (the four placements of k relative to i and j: both at or left of k, both
// right, a left and b right, b left and a right), with the positive state
// recurrences (the subset states of Sec. 4.2 for l = 3, decay mu per step)
//     X_a(t) = mu X_a(t-1) + a_t,
//     X_ab(t) = mu X_ab(t-1) + a_t (mu X_b(t-1) + b_t) + b_t mu X_a(t-1),
// and Y the mirror images from the right.  The second dimension uses the same
// recurrences with vectors over the first index, the product a_t b_t replaced
// by the one-dimensional product along the first index, FTVP1(a, b) (bilinear
// in a and b): Algorithm 6's six class sums are the six such products per
// column below.  Everything is a sum of positive terms (no cancellation); FP64
// in the linear domain, so phi and psi should be scaled to moderate values.
//
// GPU layout: phase 1 scans the columns (one thread per first index), phase 2
// runs the 6 M one-dimensional products of length N (one thread each), phase
// 3 runs the column recurrences and the combine (one thread per first index).
// Arrays are column-major: element (i1, i2) at i1 + N i2.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "mmot_internal.cuh"

namespace {

// one-dimensional product of length n (stride 1): out_k = sum_{i,j} mu^{max-min} a_i b_j
__device__ void ftvp1_dev(int n, const double *a, const double *b, double mu, double *out, double *scr)
{
    // forward states at k (inclusive): X_a, X_b, X_ab into scr[0..3n)
    double xa = 0.0, xb = 0.0, xab = 0.0;
    for (int t = 0; t < n; ++t) {
        const double at = a[t], bt = b[t];
        xab = mu * xab + at * (mu * xb + bt) + bt * mu * xa;
        xa = mu * xa + at;
        xb = mu * xb + bt;
        scr[t] = xa;
        scr[n + t] = xb;
        scr[2 * n + t] = xab;
    }
    // backward states at k+1 and the combine
    double ya = 0.0, yb = 0.0, yab = 0.0;
    for (int k = n - 1; k >= 0; --k) {
        out[k] = scr[2 * n + k] + mu * (yab + scr[k] * yb + scr[n + k] * ya);
        const double at = a[k], bt = b[k];
        yab = mu * yab + at * (mu * yb + bt) + bt * mu * ya;
        ya = mu * ya + at;
        yb = mu * yb + bt;
    }
}

// phase 1: column scans Xphi, Xpsi (forward, inclusive) and Yphi, Ypsi
// (backward, inclusive) along the second index, mu2 per step
__global__ void k_ftvp2d_scan(int N, int M, double mu2, const double *phi, const double *psi, double *Xf, double *Xs,
                              double *Yf, double *Ys)
{
    const int i1 = blockIdx.x * blockDim.x + threadIdx.x;
    if (i1 >= N) return;
    double xf = 0.0, xs = 0.0;
    for (int t = 0; t < M; ++t) {
        const size_t u = (size_t)i1 + (size_t)N * t;
        xf = mu2 * xf + phi[u];
        xs = mu2 * xs + psi[u];
        Xf[u] = xf;
        Xs[u] = xs;
    }
    double yf = 0.0, ys = 0.0;
    for (int t = M - 1; t >= 0; --t) {
        const size_t u = (size_t)i1 + (size_t)N * t;
        yf = mu2 * yf + phi[u];
        ys = mu2 * ys + psi[u];
        Yf[u] = yf;
        Ys[u] = ys;
    }
}

// phase 2: per column t the six products along the first index
//   S1 = FTVP1(phi_t, Xpsi_t)            S2 = FTVP1(mu2 Xphi_{t-1}, psi_t)
//   R1 = FTVP1(phi_t, Ypsi_t)            R2 = FTVP1(mu2 Yphi_{t+1}, psi_t)
//   C3 = FTVP1(Xphi_t, Ypsi_{t+1})       C4 = FTVP1(Yphi_{t+1}, Xpsi_t)
// (the factor mu2 of S2 and R2 is applied to the result: FTVP1 is linear)
__global__ void k_ftvp2d_cols(int N, int M, double mu1, double mu2, const double *phi, const double *psi,
                              const double *Xf, const double *Xs, const double *Yf, const double *Ys, double *zero,
                              double *out6, double *scr)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= 6 * M) return;
    const int p = id / M, t = id % M;
    const size_t c = (size_t)N * t;
    const double *a = nullptr, *b = nullptr;
    double f = 1.0;
    switch (p) {
    case 0: a = phi + c; b = Xs + c; break;
    case 1: a = (t > 0) ? Xf + c - N : zero; b = psi + c; f = mu2; break;
    case 2: a = phi + c; b = Ys + c; break;
    case 3: a = (t + 1 < M) ? Yf + c + N : zero; b = psi + c; f = mu2; break;
    case 4: a = Xf + c; b = (t + 1 < M) ? Ys + c + N : zero; break;
    default: a = (t + 1 < M) ? Yf + c + N : zero; b = Xs + c; break;
    }
    double *o = out6 + ((size_t)p * M + t) * N;
    ftvp1_dev(N, a, b, mu1, o, scr + (size_t)id * 3 * N);
    if (f != 1.0)
        for (int k = 0; k < N; ++k) o[k] *= f;
}

// phase 3: X_ab(t) = mu2 X_ab(t-1) + S1(t) + S2(t), Y_ab(t) = mu2 Y_ab(t+1) +
// R1(t) + R2(t), J(., t) = X_ab(t) + mu2 (Y_ab(t+1) + C3(t) + C4(t))
__global__ void k_ftvp2d_comb(int N, int M, double mu2, const double *out6, double *Yab, double *J)
{
    const int k1 = blockIdx.x * blockDim.x + threadIdx.x;
    if (k1 >= N) return;
    auto S = [&](int p, int t) { return out6[((size_t)p * M + t) * N + k1]; };
    double y = 0.0;
    for (int t = M - 1; t >= 0; --t) {
        Yab[(size_t)k1 + (size_t)N * t] = y;   // Y_ab(t+1)
        y = mu2 * y + S(2, t) + S(3, t);
    }
    double x = 0.0;
    for (int t = 0; t < M; ++t) {
        x = mu2 * x + S(0, t) + S(1, t);
        J[(size_t)k1 + (size_t)N * t] = x + mu2 * (Yab[(size_t)k1 + (size_t)N * t] + S(4, t) + S(5, t));
    }
}

mmot_status ftvp_err(mmot_status st, const char *fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return mmot::set_error(st, buf);
}

bool is_dev(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" mmot_status mmot_ftvp2d(int64_t N, int64_t M, const double *phi, const double *psi, double lambda1,
                                   double lambda2, double *out, void *cuda_stream)
{
    if (N < 1 || M < 1 || N > (1 << 20) || M > (1 << 20) || N * M > ((int64_t)1 << 28))
        return ftvp_err(MMOT_ERR_INVALID_ARG, "mmot_ftvp2d: N = %lld, M = %lld out of range", (long long)N,
                                  (long long)M);
    if (!phi || !psi || !out) return ftvp_err(MMOT_ERR_INVALID_ARG, "mmot_ftvp2d: NULL array");
    if (!(lambda1 >= 0.0 && lambda1 < 1.0) || !(lambda2 >= 0.0 && lambda2 < 1.0))
        return ftvp_err(MMOT_ERR_INVALID_ARG, "mmot_ftvp2d: lambda must lie in [0, 1)");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t nm = (size_t)N * (size_t)M;
    const size_t bytes = sizeof(double) * (nm * 13 + (size_t)N + 18 * (size_t)M * (size_t)N);
    double *buf = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return ftvp_err(MMOT_ERR_OOM, "mmot_ftvp2d: cudaMalloc of %zu bytes failed", bytes);
    }
    double *dphi = buf, *dpsi = buf + nm, *Xf = buf + 2 * nm, *Xs = buf + 3 * nm, *Yf = buf + 4 * nm,
           *Ys = buf + 5 * nm, *out6 = buf + 6 * nm, *Yab = buf + 12 * nm, *zero = buf + 13 * nm,
           *scr = zero + N;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    chk(cudaMemcpyAsync(dphi, phi, sizeof(double) * nm, is_dev(phi) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        st));
    chk(cudaMemcpyAsync(dpsi, psi, sizeof(double) * nm, is_dev(psi) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        st));
    chk(cudaMemsetAsync(zero, 0, sizeof(double) * N, st));
    const double mu1 = lambda1 * lambda1, mu2 = lambda2 * lambda2;
    const int n = (int)N, m = (int)M;
    if (e == cudaSuccess) {
        k_ftvp2d_scan<<<(n + 127) / 128, 128, 0, st>>>(n, m, mu2, dphi, dpsi, Xf, Xs, Yf, Ys);
        chk(cudaGetLastError());
        k_ftvp2d_cols<<<(6 * m + 127) / 128, 128, 0, st>>>(n, m, mu1, mu2, dphi, dpsi, Xf, Xs, Yf, Ys, zero, out6,
                                                            scr);
        chk(cudaGetLastError());
        double *J = is_dev(out) ? out : dphi;   // dphi is free after phase 2
        k_ftvp2d_comb<<<(n + 127) / 128, 128, 0, st>>>(n, m, mu2, out6, Yab, J);
        chk(cudaGetLastError());
        if (J != out) chk(cudaMemcpyAsync(out, J, sizeof(double) * nm, cudaMemcpyDeviceToHost, st));
    }
    chk(cudaStreamSynchronize(st));
    cudaFree(buf);
    if (e != cudaSuccess) return ftvp_err(MMOT_ERR_CUDA, "mmot_ftvp2d: %s", cudaGetErrorString(e));
    return MMOT_OK;
}
