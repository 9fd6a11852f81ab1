// construct.cu -- plan-time construction of (h_k, w_k) from a sampled
// time-varying impulse response (TVIR), on the GPU: the L2 projection of
// every row T(x, .) onto the periodic B-splines B_{alpha,m}(. - k/m) of order
// alpha = 1 (hats), 2 or 3 (Definition 2.2, Corollary 4.3).
//
//   w_k[j]  = B_{alpha,m}(j/n - k/m)                  (periodic B-splines)
//   R[d][k] = sum_j T[d][j] w_k[j]                    (right-hand sides, FP64 sums)
//   G[k][l] = sum_j w_k[j] w_l[j]                     (Gram matrix, host, FP64)
//   h_k[d]  = sum_l (G^{-1})[k][l] R[d][l]            (FP64 sums)
//
// so that T(x_d, y_j) ~ sum_k h_k[d] w_k[j], i.e. the kernel K(x, y) =
// T(x - y, y) is approximated by sum_k h_k(x - y) w_k(y), the expansion of
// Eq. 1.4 that a plan applies.  This is a construction step, not part of the
// apply: it allocates temporary buffers and synchronises the stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pce.h"
#include "plan.h"

using pce_rt::fail;

namespace {

// B_{alpha,1}(u): the centred cardinal B-spline of order alpha (Definition 2.2
// on unit knot spacing: the (alpha + 1)-fold convolution of the indicator of
// [-1/2, 1/2]), as its piecewise polynomial; B_{alpha,m}(t) = B_{alpha,1}(m t).
__device__ double cardinal_bspline(int alpha, double u) {
    const double a = fabs(u);
    if (alpha == 1) return fmax(0.0, 1.0 - a);
    if (alpha == 2) return a <= 0.5 ? 0.75 - a * a : (a <= 1.5 ? 0.5 * (1.5 - a) * (1.5 - a) : 0.0);
    return a <= 1.0 ? 2.0 / 3.0 - a * a + 0.5 * a * a * a : (a <= 2.0 ? (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0 : 0.0);
}

// periodic B-splines of order alpha at the m nodes k/m on n samples, as the plan
// receives them (float32): w[k][j] = B_{alpha,m}(j/n - k/m)
__global__ void k_bsplines(int n, int m, int alpha, float* w) {
    const long long total = (long long)m * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / n), j = (int)(i % n);
        double t = (double)j / n - (double)k / m;
        t -= rint(t);   // periodic distance in [-1/2, 1/2]
        w[i] = (float)cardinal_bspline(alpha, m * t);
    }
}

// R[d][k] = sum_j T[d][j] w_k[j] over the support of w_k (|j/n - k/m| < (alpha + 1) / (2m))
__global__ void k_proj_rhs(const float* __restrict__ T, const float* __restrict__ w, int n, int m, int alpha,
                           double* __restrict__ R) {
    const long long total = (long long)n * m;
    // samples on each side of the node
    const int half = (int)(((long long)(alpha + 1) * n + 2 * m - 1) / (2 * m)) + 2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int d = (int)(i / m), k = (int)(i % m);
        const int c = (int)(((long long)k * n) / m);
        const int span = min(n, 2 * half + 1);
        double s = 0.0;
        for (int t = 0; t < span; ++t) {
            int j = c - half + t;
            j %= n;
            if (j < 0) j += n;
            const float wk = w[(long long)k * n + j];
            if (wk != 0.f) s += (double)T[(long long)d * n + j] * (double)wk;
        }
        R[i] = s;
    }
}

// h[k][d] = sum_l Ginv[k][l] R[d][l]
__global__ void k_proj_solve(const double* __restrict__ R, const double* __restrict__ Ginv, int n, int m,
                             float* __restrict__ h) {
    const long long total = (long long)n * m;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / n), d = (int)(i % n);
        double s = 0.0;
        for (int l = 0; l < m; ++l) s += Ginv[(long long)k * m + l] * R[(long long)d * m + l];
        h[i] = (float)s;
    }
}

unsigned grid_of(long long total) {
    return (unsigned)std::max<long long>(1, std::min<long long>((total + 255) / 256, 1 << 16));
}

// Inverse of a symmetric positive definite m x m matrix (Gauss-Jordan with
// partial pivoting, FP64).  Returns false if singular.
bool invert(std::vector<double>& a, int m, std::vector<double>& inv) {
    inv.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) inv[(size_t)i * m + i] = 1.0;
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < m; ++r)
            if (std::fabs(a[(size_t)r * m + c]) > std::fabs(a[(size_t)piv * m + c])) piv = r;
        if (std::fabs(a[(size_t)piv * m + c]) < 1e-300) return false;
        if (piv != c)
            for (int j = 0; j < m; ++j) {
                std::swap(a[(size_t)c * m + j], a[(size_t)piv * m + j]);
                std::swap(inv[(size_t)c * m + j], inv[(size_t)piv * m + j]);
            }
        const double d = a[(size_t)c * m + c];
        for (int j = 0; j < m; ++j) {
            a[(size_t)c * m + j] /= d;
            inv[(size_t)c * m + j] /= d;
        }
        for (int r = 0; r < m; ++r) {
            if (r == c) continue;
            const double f = a[(size_t)r * m + c];
            if (f == 0.0) continue;
            for (int j = 0; j < m; ++j) {
                a[(size_t)r * m + j] -= f * a[(size_t)c * m + j];
                inv[(size_t)r * m + j] -= f * inv[(size_t)c * m + j];
            }
        }
    }
    return true;
}

}  // namespace

extern "C" pce_status pce_construct_projection_bspline_1d(const float* T, int n, int m, int alpha, float* h_out,
                                                          float* w_out, void* stream) {
    if (alpha < 1 || alpha > 3) return fail(PCE_ERR_INVALID, "alpha must be 1, 2 or 3 (got %d)", alpha);
    if (n < 16 || n > (1 << 18)) return fail(PCE_ERR_INVALID, "n must be in [16, 262144] (got %d)", n);
    if (m < alpha + 2 || m > std::min(n, 512))
        return fail(PCE_ERR_INVALID, "m must be in [alpha + 2, min(n, 512)] (got %d, alpha %d)", m, alpha);
    if (!pce_rt::is_device_ptr(T) || !pce_rt::is_device_ptr(h_out) || !pce_rt::is_device_ptr(w_out))
        return fail(PCE_ERR_INVALID, "T, h_out and w_out must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* R = nullptr;
    double* Gi = nullptr;
    auto cleanup = [&]() {
        if (R) cudaFree(R);
        if (Gi) cudaFree(Gi);
    };
    cudaError_t e = cudaMalloc(&R, sizeof(double) * (size_t)n * m);
    if (e == cudaSuccess) e = cudaMalloc(&Gi, sizeof(double) * (size_t)m * m);
    if (e == cudaSuccess) {
        k_bsplines<<<grid_of((long long)m * n), 256, 0, s>>>(n, m, alpha, w_out);
        k_proj_rhs<<<grid_of((long long)n * m), 256, 0, s>>>(T, w_out, n, m, alpha, R);
        e = cudaGetLastError();
    }
    // Gram matrix of the float32 hats the plan will use, in FP64 on the host
    std::vector<float> wh((size_t)m * n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(wh.data(), w_out, sizeof(float) * wh.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cleanup();
        return fail(e == cudaErrorMemoryAllocation ? PCE_ERR_OOM : PCE_ERR_CUDA, "projection set-up: %s",
                    cudaGetErrorString(e));
    }
    // a sample j meets the B-splines whose nodes are within (alpha + 1) / (2m) of
    // j/n: k in floor(j m / n) - r .. + r + 1 (mod m), r = (alpha + 2) / 2, covers them all
    const int r = (alpha + 2) / 2;
    std::vector<double> G((size_t)m * m, 0.0);
    for (int j = 0; j < n; ++j) {
        const int k0 = (int)(((long long)j * m) / n);
        int ks[8], nk = 0;
        for (int dk = -r; dk <= r + 1; ++dk) {
            const int k = ((k0 + dk) % m + m) % m;
            bool seen = false;
            for (int t = 0; t < nk; ++t) seen |= ks[t] == k;
            if (!seen && wh[(size_t)k * n + j] != 0.f) ks[nk++] = k;
        }
        for (int a = 0; a < nk; ++a)
            for (int b = 0; b < nk; ++b)
                G[(size_t)ks[a] * m + ks[b]] += (double)wh[(size_t)ks[a] * n + j] * (double)wh[(size_t)ks[b] * n + j];
    }
    std::vector<double> Ginv;
    if (!invert(G, m, Ginv)) {
        cleanup();
        return fail(PCE_ERR_INVALID, "the Gram matrix of %d B-splines on %d samples is singular", m, n);
    }
    e = cudaMemcpyAsync(Gi, Ginv.data(), sizeof(double) * Ginv.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_proj_solve<<<grid_of((long long)n * m), 256, 0, s>>>(R, Gi, n, m, h_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return fail(PCE_ERR_CUDA, "projection: %s", cudaGetErrorString(e));
    return PCE_OK;
}

extern "C" pce_status pce_construct_projection_1d(const float* T, int n, int m, float* h_out, float* w_out,
                                                  void* stream) {
    return pce_construct_projection_bspline_1d(T, n, m, 1, h_out, w_out, stream);
}

// ---------------------------------------------------------------------------
// 2D: the L2 projection of every row T(x_d, .) of a 2D TVIR onto the
// tensor-product hats B_k(y) = B_{1,gy}(y1 - i/gy) B_{1,gx}(y2 - l/gx), k = i gx + l
// (Corollary 4.3 with the windows of the 2D workloads).  The Gram matrix of
// product windows is the Kronecker product of the 1D Gram matrices, so its
// inverse is the Kronecker product of two small inverses (host, FP64).
//
//   R[k][s]  = sum_j T[j][s] wy_k[row j] wx_k[col j]    (device, FP64 sums over the window's box)
//   h_k[d_s] = sum_k' (Gy^-1 (x) Gx^-1)[k][k'] R[k'][s]  (device, FP64)
//
// with s = (a, b) a position of the shift window and d_s = (a - sy/2, b - sx/2).
// ---------------------------------------------------------------------------
namespace {

// wy[k][r] = B_{1,gy}(r/ny - i/gy), wx[k][c] = B_{1,gx}(c/nx - l/gx), k = i gx + l
__global__ void k_hat_factors(int ny, int nx, int gy, int gx, float* wy, float* wx) {
    const int m = gy * gx;
    const long long total = (long long)m * (ny + nx);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / (ny + nx)), q = (int)(e % (ny + nx));
        const int i = k / gx, l = k % gx;
        if (q < ny) {
            double t = (double)q / ny - (double)i / gy;
            t -= rint(t);
            wy[(long long)k * ny + q] = (float)cardinal_bspline(1, gy * t);
        } else {
            const int c = q - ny;
            double t = (double)c / nx - (double)l / gx;
            t -= rint(t);
            wx[(long long)k * nx + c] = (float)cardinal_bspline(1, gx * t);
        }
    }
}

// R[k][s] = sum over the box of window k of T[j][s] wy_k[r] wx_k[c] (FP64), one thread per (k, s)
__global__ void k_proj2d_rhs(const float* __restrict__ T, int ny, int nx, int S, int gy, int gx,
                             const float* __restrict__ wy, const float* __restrict__ wx, double* __restrict__ R) {
    const int m = gy * gx;
    const long long total = (long long)m * S;
    const int hy = ny / gy + 2, hx = nx / gx + 2;   // samples on each side of a node
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / S), sidx = (int)(e % S);
        const int i = k / gx, l = k % gx;
        const int ry = (int)(((long long)i * ny) / gy), cx = (int)(((long long)l * nx) / gx);
        const int spy = min(ny, 2 * hy + 1), spx = min(nx, 2 * hx + 1);
        double acc = 0.0;
        for (int tr = 0; tr < spy; ++tr) {
            int r = (ry - hy + tr) % ny;
            if (r < 0) r += ny;
            const float fy = wy[(long long)k * ny + r];
            if (fy == 0.f) continue;
            for (int tc = 0; tc < spx; ++tc) {
                int c = (cx - hx + tc) % nx;
                if (c < 0) c += nx;
                const float fx = wx[(long long)k * nx + c];
                if (fx == 0.f) continue;
                acc += (double)T[((long long)r * nx + c) * S + sidx] * (double)fy * (double)fx;
            }
        }
        R[e] = acc;
    }
}

// h[k][d_s] = sum_k' Ginv[k][k'] R[k'][s]; the rest of h was zeroed
__global__ void k_proj2d_solve(const double* __restrict__ R, const double* __restrict__ Ginv, int m, int S, int ny,
                               int nx, int sy, int sx, float* __restrict__ h) {
    const long long total = (long long)m * S;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / S), sidx = (int)(e % S);
        double acc = 0.0;
        for (int kk = 0; kk < m; ++kk) acc += Ginv[(long long)k * m + kk] * R[(long long)kk * S + sidx];
        const int a = sidx / sx, b = sidx % sx;
        int dr = (a - sy / 2) % ny, dc = (b - sx / 2) % nx;
        if (dr < 0) dr += ny;
        if (dc < 0) dc += nx;
        h[((long long)k * ny + dr) * nx + dc] = (float)acc;
    }
}

// Gram matrix of the float32 1D hats of one axis (FP64), from their device copy
bool gram_1d(const std::vector<float>& w, int g, int n, std::vector<double>& G) {
    G.assign((size_t)g * g, 0.0);
    for (int a = 0; a < g; ++a)
        for (int b = 0; b < g; ++b) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += (double)w[(size_t)a * n + j] * (double)w[(size_t)b * n + j];
            G[(size_t)a * g + b] = s;
        }
    return true;
}

}  // namespace

extern "C" pce_status pce_construct_projection_2d(const float* T, int ny, int nx, int sy, int sx, int gy, int gx,
                                                  float* h_out, float* wy_out, float* wx_out, void* stream) {
    if (ny < 4 || nx < 4 || ny > 4096 || nx > 4096)
        return fail(PCE_ERR_INVALID, "ny and nx must be in [4, 4096] (got %d, %d)", ny, nx);
    if (sy < 1 || sy > ny || sx < 1 || sx > nx)
        return fail(PCE_ERR_INVALID, "the shift window %d x %d must lie in [1, ny] x [1, nx]", sy, sx);
    if (gy < 2 || gx < 2 || gy > std::min(ny, 64) || gx > std::min(nx, 64))
        return fail(PCE_ERR_INVALID, "the node grid %d x %d must lie in [2, min(n, 64)] per axis", gy, gx);
    if (!pce_rt::is_device_ptr(T) || !pce_rt::is_device_ptr(h_out) || !pce_rt::is_device_ptr(wy_out) ||
        !pce_rt::is_device_ptr(wx_out))
        return fail(PCE_ERR_INVALID, "T, h_out, wy_out and wx_out must be device pointers");
    const int m = gy * gx, S = sy * sx;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* R = nullptr;
    double* Gi = nullptr;
    auto cleanup = [&]() {
        if (R) cudaFree(R);
        if (Gi) cudaFree(Gi);
    };
    cudaError_t e = cudaMalloc(&R, sizeof(double) * (size_t)m * S);
    if (e == cudaSuccess) e = cudaMalloc(&Gi, sizeof(double) * (size_t)m * m);
    if (e == cudaSuccess) e = cudaMemsetAsync(h_out, 0, sizeof(float) * (size_t)m * ny * nx, s);
    if (e == cudaSuccess) {
        k_hat_factors<<<grid_of((long long)m * (ny + nx)), 256, 0, s>>>(ny, nx, gy, gx, wy_out, wx_out);
        k_proj2d_rhs<<<grid_of((long long)m * S), 256, 0, s>>>(T, ny, nx, S, gy, gx, wy_out, wx_out, R);
        e = cudaGetLastError();
    }
    // the 1D hats of each axis (rows k = i gx of wy, k = l of wx) for the Gram matrices
    std::vector<float> hy((size_t)m * ny), hx((size_t)m * nx);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hy.data(), wy_out, sizeof(float) * hy.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hx.data(), wx_out, sizeof(float) * hx.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cleanup();
        return fail(e == cudaErrorMemoryAllocation ? PCE_ERR_OOM : PCE_ERR_CUDA, "2D projection set-up: %s",
                    cudaGetErrorString(e));
    }
    std::vector<float> by((size_t)gy * ny), bx((size_t)gx * nx);
    for (int i = 0; i < gy; ++i)
        std::copy(hy.begin() + (size_t)(i * gx) * ny, hy.begin() + (size_t)(i * gx + 1) * ny, by.begin() + (size_t)i * ny);
    std::copy(hx.begin(), hx.begin() + (size_t)gx * nx, bx.begin());
    std::vector<double> Gy, Gx, Gyi, Gxi;
    gram_1d(by, gy, ny, Gy);
    gram_1d(bx, gx, nx, Gx);
    if (!invert(Gy, gy, Gyi) || !invert(Gx, gx, Gxi)) {
        cleanup();
        return fail(PCE_ERR_INVALID, "the Gram matrix of the %d x %d hats on %d x %d samples is singular", gy, gx,
                    ny, nx);
    }
    std::vector<double> Ginv((size_t)m * m);
    for (int i = 0; i < gy; ++i)
        for (int l = 0; l < gx; ++l)
            for (int i2 = 0; i2 < gy; ++i2)
                for (int l2 = 0; l2 < gx; ++l2)
                    Ginv[(size_t)(i * gx + l) * m + (i2 * gx + l2)] = Gyi[(size_t)i * gy + i2] * Gxi[(size_t)l * gx + l2];
    e = cudaMemcpyAsync(Gi, Ginv.data(), sizeof(double) * Ginv.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_proj2d_solve<<<grid_of((long long)m * S), 256, 0, s>>>(R, Gi, m, S, ny, nx, sy, sx, h_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return fail(PCE_ERR_CUDA, "2D projection: %s", cudaGetErrorString(e));
    return PCE_OK;
}

// ---------------------------------------------------------------------------
// Truncated SVD of the TVIR (Section 5.1): T(x, y) ~ sum_k sigma_k f_k(x) e_k(y)
// with h_k = sigma_k f_k and w_k = e_k, the best rank-m approximation.  The
// leading singular subspace is found by the randomised range finder with
// power iterations of Halko, Martinsson and Tropp (2011), the method the
// paper's operation count refers to:
//
//   Y = T Omega                     (Omega: n x l Gaussian, l = m + oversampling)
//   Q = orth(Y);  q times: Q = orth(T orth(T^t Q))
//   B^t = T^t Q                     (n x l; B = Q^t T)
//   B^t = Q2 R                      (host, FP64 Householder QR)
//   R = U_R diag(sigma) V_R^t       (host, FP64 one-sided Jacobi)
//   f_k = (Q V_R)_k,  e_k = (Q2 U_R)_k
//
// (no Gram matrix of B is formed, so small singular values keep their
// relative accuracy and the e_k are orthonormal to rounding)
//
// orth() is the Q factor of a Householder QR (host, FP64): it keeps all l
// directions, so singular values down to the rounding level of T survive.
// The products with T are FP64 sums of the float32 T on the device.
// ---------------------------------------------------------------------------
namespace {

// SplitMix64 (Steele, Lea and Flood, 2014): the counter-based generator of
// the test matrix; its output for counter c is mix(seed + (c + 1) * gamma).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// X[i][c] ~ N(0, 1) by the Box-Muller transform of two SplitMix64 draws
__global__ void k_gaussian(long long total, unsigned long long seed, double* __restrict__ X) {
    const unsigned long long gamma = 0x9E3779B97F4A7C15ull;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long a = splitmix64(seed + (2ull * i + 1ull) * gamma);
        const unsigned long long b = splitmix64(seed + (2ull * i + 2ull) * gamma);
        const double u1 = ((double)(a >> 11) + 1.0) * 0x1.0p-53;   // (0, 1]
        const double u2 = (double)(b >> 11) * 0x1.0p-53;           // [0, 1)
        X[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
}

// Y = T X (TRANS = false) or Y = T^t X (TRANS = true); T [n][n] float32,
// X, Y [n][l] FP64.  One thread per output element; the l threads of a row
// share the T element (broadcast) and read X coalesced.
template <bool TRANS>
__global__ void k_tvir_mul(const float* __restrict__ T, const double* __restrict__ X, int n, int l,
                           double* __restrict__ Y) {
    const long long total = (long long)n * l;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / l), c = (int)(e % l);
        double s = 0.0;
        if (TRANS) {
            for (int i = 0; i < n; ++i) s += (double)__ldg(&T[(long long)i * n + r]) * X[(long long)i * l + c];
        } else {
            const float* Tr = T + (long long)r * n;
            for (int j = 0; j < n; ++j) s += (double)__ldg(&Tr[j]) * X[(long long)j * l + c];
        }
        Y[e] = s;
    }
}

// Z = Y M, Y [n][l], M [l][l2], Z [n][l2]
__global__ void k_right_mul(const double* __restrict__ Y, const double* __restrict__ M, int n, int l, int l2,
                            double* __restrict__ Z) {
    const long long total = (long long)n * l2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / l2), c = (int)(e % l2);
        double s = 0.0;
        for (int a = 0; a < l; ++a) s += Y[(long long)i * l + a] * M[a * l2 + c];
        Z[e] = s;
    }
}

// out[k][i] = scale[k] * Z[i][k] (float32), Z [n][m]
__global__ void k_terms_out(const double* __restrict__ Z, const double* __restrict__ scale, int n, int m,
                            float* __restrict__ out) {
    const long long total = (long long)n * m;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), i = (int)(e % n);
        out[e] = (float)(scale[k] * Z[(long long)i * m + k]);
    }
}

}  // namespace

namespace {

// Householder QR of A (n x l, n >= l, row-major, destroyed) (Golub and Van
// Loan, Section 5.2): A = Q2 R with Q2 (n x l) orthonormal columns, R (l x l)
// upper triangular.
void householder_qr(std::vector<double>& A, int n, int l, std::vector<double>& Q2, std::vector<double>& R) {
    std::vector<std::vector<double>> vs(l);
    std::vector<double> beta(l, 0.0);
    for (int j = 0; j < l; ++j) {
        double nrm = 0.0;
        for (int i = j; i < n; ++i) nrm += A[(size_t)i * l + j] * A[(size_t)i * l + j];
        nrm = std::sqrt(nrm);
        std::vector<double>& v = vs[j];
        v.assign(n - j, 0.0);
        for (int i = j; i < n; ++i) v[i - j] = A[(size_t)i * l + j];
        if (nrm == 0.0) continue;   // zero column: no reflection
        const double x0 = v[0];
        v[0] = x0 + (x0 >= 0.0 ? nrm : -nrm);
        double vv = 0.0;
        for (double x : v) vv += x * x;
        beta[j] = 2.0 / vv;
        for (int c = j; c < l; ++c) {   // A[j:, c] -= beta v (v . A[j:, c])
            double d = 0.0;
            for (int i = j; i < n; ++i) d += v[i - j] * A[(size_t)i * l + c];
            d *= beta[j];
            for (int i = j; i < n; ++i) A[(size_t)i * l + c] -= d * v[i - j];
        }
    }
    R.assign((size_t)l * l, 0.0);
    for (int i = 0; i < l; ++i)
        for (int c = i; c < l; ++c) R[(size_t)i * l + c] = A[(size_t)i * l + c];
    // Q2 = H_0 H_1 ... H_{l-1} [I; 0], accumulated from the last reflection
    Q2.assign((size_t)n * l, 0.0);
    for (int i = 0; i < l; ++i) Q2[(size_t)i * l + i] = 1.0;
    for (int j = l - 1; j >= 0; --j) {
        if (beta[j] == 0.0) continue;
        const std::vector<double>& v = vs[j];
        for (int c = 0; c < l; ++c) {
            double d = 0.0;
            for (int i = j; i < n; ++i) d += v[i - j] * Q2[(size_t)i * l + c];
            d *= beta[j];
            for (int i = j; i < n; ++i) Q2[(size_t)i * l + c] -= d * v[i - j];
        }
    }
}

// One-sided Jacobi SVD of a square R (l x l) (Hestenes; Demmel and Veselic,
// 1992): plane rotations from the right make the columns of R V mutually
// orthogonal; sigma_c = |(R V)_c|, U_R = (R V) diag(1/sigma), V_R = V.
// Sweeps until every pair is orthogonal to 1e-15 relative, at most 60.
void one_sided_jacobi(std::vector<double> R, int l, std::vector<double>& sv, std::vector<double>& U,
                      std::vector<double>& V) {
    V.assign((size_t)l * l, 0.0);
    for (int i = 0; i < l; ++i) V[(size_t)i * l + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        bool rotated = false;
        for (int p = 0; p < l; ++p)
            for (int q = p + 1; q < l; ++q) {
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < l; ++i) {
                    const double rp = R[(size_t)i * l + p], rq = R[(size_t)i * l + q];
                    al += rp * rp;
                    be += rq * rq;
                    ga += rp * rq;
                }
                if (ga == 0.0 || std::fabs(ga) <= 1e-15 * std::sqrt(al * be)) continue;
                rotated = true;
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int i = 0; i < l; ++i) {
                    const double rp = R[(size_t)i * l + p], rq = R[(size_t)i * l + q];
                    R[(size_t)i * l + p] = c * rp - s * rq;
                    R[(size_t)i * l + q] = s * rp + c * rq;
                    const double vp = V[(size_t)i * l + p], vq = V[(size_t)i * l + q];
                    V[(size_t)i * l + p] = c * vp - s * vq;
                    V[(size_t)i * l + q] = s * vp + c * vq;
                }
            }
        if (!rotated) break;
    }
    sv.assign(l, 0.0);
    U.assign((size_t)l * l, 0.0);
    for (int c = 0; c < l; ++c) {
        double nrm = 0.0;
        for (int i = 0; i < l; ++i) nrm += R[(size_t)i * l + c] * R[(size_t)i * l + c];
        sv[c] = std::sqrt(nrm);
        if (sv[c] > 0.0)
            for (int i = 0; i < l; ++i) U[(size_t)i * l + c] = R[(size_t)i * l + c] / sv[c];
    }
}

}  // namespace

namespace {

// Y [n][l] (device) <- the Q factor of its Householder QR, computed on the
// host in FP64; returns false on a CUDA error (in e).
bool orth(double* Y, int n, int l, cudaStream_t s, cudaError_t& e) {
    std::vector<double> a((size_t)n * l), q, r;
    e = cudaMemcpyAsync(a.data(), Y, sizeof(double) * a.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return false;
    householder_qr(a, n, l, q, r);
    e = cudaMemcpyAsync(Y, q.data(), sizeof(double) * q.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // q must outlive the copy
    return e == cudaSuccess;
}

}  // namespace

extern "C" pce_status pce_construct_svd_1d(const float* T, int n, int m, int oversample, int power_iters,
                                           unsigned long long seed, float* h_out, float* w_out, float* sigma_out,
                                           void* stream) {
    if (n < 16 || n > 8192) return fail(PCE_ERR_INVALID, "n must be in [16, 8192] (got %d)", n);
    if (m < 1 || m > std::min(n, 256)) return fail(PCE_ERR_INVALID, "m must be in [1, min(n, 256)] (got %d)", m);
    if (oversample < 0 || oversample > 256 || power_iters < 0 || power_iters > 16)
        return fail(PCE_ERR_INVALID, "oversample must be in [0, 256] and power_iters in [0, 16]");
    if (!pce_rt::is_device_ptr(T) || !pce_rt::is_device_ptr(h_out) || !pce_rt::is_device_ptr(w_out) ||
        (sigma_out && !pce_rt::is_device_ptr(sigma_out)))
        return fail(PCE_ERR_INVALID, "T, h_out, w_out and sigma_out must be device pointers");
    const int l = std::min(n, m + oversample);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *Y = nullptr, *Z = nullptr, *tmp = nullptr, *M = nullptr, *sc = nullptr;
    auto cleanup = [&]() {
        for (double* q : {Y, Z, tmp, M, sc})
            if (q) cudaFree(q);
    };
    const size_t nl = (size_t)n * l;
    cudaError_t e = cudaMalloc(&Y, sizeof(double) * nl);
    if (e == cudaSuccess) e = cudaMalloc(&Z, sizeof(double) * nl);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, sizeof(double) * nl);
    if (e == cudaSuccess) e = cudaMalloc(&M, sizeof(double) * (size_t)l * l);
    if (e == cudaSuccess) e = cudaMalloc(&sc, sizeof(double) * (size_t)std::max(l, m));
    if (e != cudaSuccess) {
        cleanup();
        return fail(e == cudaErrorMemoryAllocation ? PCE_ERR_OOM : PCE_ERR_CUDA, "svd set-up: %s",
                    cudaGetErrorString(e));
    }
    // range finder: Y = T Omega, then power iterations
    k_gaussian<<<grid_of((long long)nl), 256, 0, s>>>((long long)nl, seed, Z);
    k_tvir_mul<false><<<grid_of((long long)nl), 256, 0, s>>>(T, Z, n, l, Y);
    e = cudaGetLastError();
    bool ok = e == cudaSuccess && orth(Y, n, l, s, e);
    for (int it = 0; it < power_iters && ok; ++it) {
        k_tvir_mul<true><<<grid_of((long long)nl), 256, 0, s>>>(T, Y, n, l, Z);
        e = cudaGetLastError();
        ok = e == cudaSuccess && orth(Z, n, l, s, e);
        if (!ok) break;
        k_tvir_mul<false><<<grid_of((long long)nl), 256, 0, s>>>(T, Z, n, l, Y);
        e = cudaGetLastError();
        ok = e == cudaSuccess && orth(Y, n, l, s, e);
    }
    // B^t = T^t Q (into Z), brought to the host for its SVD
    std::vector<double> bt(nl);
    if (ok) {
        k_tvir_mul<true><<<grid_of((long long)nl), 256, 0, s>>>(T, Y, n, l, Z);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(bt.data(), Z, sizeof(double) * nl, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (!ok || e != cudaSuccess) {
        cleanup();
        return fail(PCE_ERR_CUDA, "svd range finder: %s", cudaGetErrorString(e));
    }
    // B^t = Q2 R (Householder), R = U_R diag(sigma) V_R^t (one-sided Jacobi), so
    // that T ~ Q B = (Q V_R) diag(sigma) (Q2 U_R)^t: f_k = (Q V_R)_k, e_k = (Q2 U_R)_k
    std::vector<double> q2, R;
    householder_qr(bt, n, l, q2, R);
    std::vector<double> sv, UR, VR;
    one_sided_jacobi(R, l, sv, UR, VR);
    std::vector<int> order(l);
    for (int i = 0; i < l; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sv[a] > sv[b]; });
    const double smax = sv[order[0]];
    std::vector<double> vm((size_t)l * m, 0.0), sig(m, 0.0);
    std::vector<float> wf((size_t)m * n, 0.f);
    std::vector<double> q2sum(l, 0.0);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < l; ++a) q2sum[a] += q2[(size_t)i * l + a];
    for (int k = 0; k < m && k < l; ++k) {
        const int c = order[k];
        if (!(sv[c] > 1e-12 * smax)) continue;   // no range left: a zero term
        // sign: sum_j e_k[j] >= 0
        double t = 0.0;
        for (int a = 0; a < l; ++a) t += q2sum[a] * UR[(size_t)a * l + c];
        const double sgn = t < 0.0 ? -1.0 : 1.0;
        sig[k] = sv[c];
        for (int a = 0; a < l; ++a) vm[(size_t)a * m + k] = sgn * VR[(size_t)a * l + c];
        for (int i = 0; i < n; ++i) {
            double x = 0.0;
            for (int a = 0; a < l; ++a) x += q2[(size_t)i * l + a] * UR[(size_t)a * l + c];
            wf[(size_t)k * n + i] = (float)(sgn * x);
        }
    }
    std::vector<float> sigf(sig.begin(), sig.end());
    // h_k = sigma_k (Q V_R)_k on the device; w_k from the host
    e = cudaMemcpyAsync(M, vm.data(), sizeof(double) * vm.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc, sig.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_right_mul<<<grid_of((long long)n * m), 256, 0, s>>>(Y, M, n, l, m, tmp);
        k_terms_out<<<grid_of((long long)n * m), 256, 0, s>>>(tmp, sc, n, m, h_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(w_out, wf.data(), sizeof(float) * wf.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && sigma_out)
        e = cudaMemcpyAsync(sigma_out, sigf.data(), sizeof(float) * m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return fail(PCE_ERR_CUDA, "svd: %s", cudaGetErrorString(e));
    return PCE_OK;
}
