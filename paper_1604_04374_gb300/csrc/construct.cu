// construct.cu -- plan-time construction of (h_k, w_k) from a sampled
// time-varying impulse response (TVIR), on the GPU: the L2 projection of
// every row T(x, .) onto the periodic hats B_{1,m}(. - k/m) (Corollary 4.3).
//
//   w_k[j]  = B_{1,m}(j/n - k/m)                      (periodic hats)
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

// periodic hat of m nodes on n samples, as the plan receives it (float32)
__global__ void k_hats(int n, int m, float* w) {
    const long long total = (long long)m * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / n), j = (int)(i % n);
        double t = (double)j / n - (double)k / m;
        t -= rint(t);   // periodic distance in [-1/2, 1/2]
        w[i] = (float)fmax(0.0, 1.0 - m * fabs(t));
    }
}

// R[d][k] = sum_j T[d][j] w_k[j] over the support of w_k (|j/n - k/m| < 1/m)
__global__ void k_proj_rhs(const float* __restrict__ T, const float* __restrict__ w, int n, int m,
                           double* __restrict__ R) {
    const long long total = (long long)n * m;
    const int half = (int)((long long)n / m) + 2;   // samples on each side of the node
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

extern "C" pce_status pce_construct_projection_1d(const float* T, int n, int m, float* h_out, float* w_out,
                                                  void* stream) {
    if (n < 16 || n > (1 << 18)) return fail(PCE_ERR_INVALID, "n must be in [16, 262144] (got %d)", n);
    if (m < 3 || m > std::min(n, 512)) return fail(PCE_ERR_INVALID, "m must be in [3, min(n, 512)] (got %d)", m);
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
        k_hats<<<grid_of((long long)m * n), 256, 0, s>>>(n, m, w_out);
        k_proj_rhs<<<grid_of((long long)n * m), 256, 0, s>>>(T, w_out, n, m, R);
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
    // a sample j meets the hats whose nodes are within 1/m of j/n: k in
    // floor(j m / n) - 1 .. + 2 (mod m) covers them all
    std::vector<double> G((size_t)m * m, 0.0);
    for (int j = 0; j < n; ++j) {
        const int k0 = (int)(((long long)j * m) / n);
        int ks[4], nk = 0;
        for (int dk = -1; dk <= 2; ++dk) {
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
        return fail(PCE_ERR_INVALID, "the Gram matrix of %d hats on %d samples is singular", m, n);
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
