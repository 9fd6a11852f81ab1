// k1d.cu -- instances of the single-CTA 1D kernels for N = 16 .. 8192.
#include "kernels.cuh"
#include "launch.h"

namespace pce {

#define PCE_1D_SIZES(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192)

int fft1d_threads(int n) {
    switch (n) {
#define X(N) case N: return Cfg1d<N>::NT;
        PCE_1D_SIZES(X)
#undef X
    }
    return 0;
}
int fft1d_smem(int n) {
    switch (n) {
#define X(N) case N: return Cfg1d<N>::SMEM;
        PCE_1D_SIZES(X)
#undef X
    }
    return 0;
}

cudaError_t prepare_cols();

cudaError_t prepare_kernels() {
    cudaError_t e = prepare_cols();
#define X(N)                                                                                   \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_fwd_1d<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                 Cfg1d<N>::SMEM);                                              \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_adj_1d<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                 Cfg1d<N>::SMEM);                                              \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_spec_1d<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                 Cfg1d<N>::SMEM);                                              \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_grad_1d<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                 Cfg1d<N>::SMEM);
    PCE_1D_SIZES(X)
#undef X
    return e;
}

cudaError_t launch_fwd_1d(int n, int batch, cudaStream_t s, const float* u, const float* w,
                          const float2* hp, int m, float* y, float scale, const float2* tw) {
    switch (n) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        k_fwd_1d<N><<<batch, Cfg1d<N>::NT, Cfg1d<N>::SMEM, s>>>(u, w, hp, m, y, scale, tw);    \
        break;
        PCE_1D_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_1d(int n, int batch, cudaStream_t s, const float* v, const float* w,
                          const float2* hp, int m, float* x, float scale, const float2* tw) {
    switch (n) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        k_adj_1d<N><<<batch, Cfg1d<N>::NT, Cfg1d<N>::SMEM, s>>>(v, w, hp, m, x, scale, tw);    \
        break;
        PCE_1D_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_spec_1d(int n, int m, cudaStream_t s, const float* h, float2* hp,
                           const float2* tw) {
    switch (n) {
#define X(N)                                                                                   \
    case N: {                                                                                  \
        const int npairs = (m + 1) / 2;                                                        \
        const int grid = (npairs + Cfg1d<N>::G - 1) / Cfg1d<N>::G;                              \
        k_spec_1d<N><<<grid, Cfg1d<N>::NT, Cfg1d<N>::SMEM, s>>>(h, m, hp, tw);                 \
        break;                                                                                 \
    }
        PCE_1D_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_grad_1d(int n, int m, cudaStream_t s, const float* u, const float* r,
                           const float* w, const float2* hp, int nb, float2* dh, float* dw,
                           float scale, int accumulate, const float2* tw) {
    switch (n) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        k_grad_1d<N><<<m, Cfg1d<N>::NT, Cfg1d<N>::SMEM, s>>>(u, r, w, hp, nb, dh, dw, scale,   \
                                                             accumulate, tw);                  \
        break;
        PCE_1D_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pce
