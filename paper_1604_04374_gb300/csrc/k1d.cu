// k1d.cu -- instances of the single-CTA 1D kernels for N = 16 .. 8192.
#include "kernels.cuh"
#include "k1d_large.cuh"
#include "wk1d.cuh"
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

#define PCE_L1_SIZES(X) X(128) X(256) X(512)

cudaError_t prepare_l1() {
    cudaError_t e = cudaSuccess;
#define X(N)                                                                                   \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k4_cols<N, kL1Win>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 ColCfg<N>::SMEM);                                             \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k4_cols<N, kL1Pair>,                                          \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<N>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k4_cols<N, kL1One>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 ColCfg<N>::SMEM);                                             \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k4_cols_inv<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                 ColCfg<N>::SMEM);                                             \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k4_cols_adj<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                 ColCfg<N>::SMEM);                                             \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k4_rows_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                 L1Rows<N>::SMEM);                                             \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k4_rows_adj<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                 L1Rows<N>::SMEM);                                             \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k4_rows_spec<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 L1Rows<N>::SMEM);
    PCE_L1_SIZES(X)
#undef X
    return e;
}

int l1_cols_per_cta(int ny) { return cols_columns_per_cta(ny); }
int l1_row_items(int nx) {
    switch (nx) {
#define X(N) case N: return L1Rows<N>::ITEMS;
        PCE_L1_SIZES(X)
#undef X
    }
    return 0;
}

cudaError_t launch_l1_cols(int ny, int mode, dim3 grid, cudaStream_t s, const float* src,
                           long long src_bstride, const float* w, int m, int nx, const float2* twN,
                           float2* G, const float2* tw) {
    switch (ny) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        if (mode == kL1Win)                                                                    \
            k4_cols<N, kL1Win><<<grid, ColCfg<N>::NT, ColCfg<N>::SMEM, s>>>(src, src_bstride, w, m, \
                                                                           nx, twN, G, tw);   \
        else if (mode == kL1Pair)                                                              \
            k4_cols<N, kL1Pair><<<grid, ColCfg<N>::NT, ColCfg<N>::SMEM, s>>>(src, src_bstride, w,  \
                                                                            m, nx, twN, G, tw); \
        else                                                                                   \
            k4_cols<N, kL1One><<<grid, ColCfg<N>::NT, ColCfg<N>::SMEM, s>>>(src, src_bstride, w, m, \
                                                                           nx, twN, G, tw);   \
        break;
        PCE_L1_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_l1_rows_fwd(int nx, dim3 grid, cudaStream_t s, const float2* G, int npairs,
                               const float2* hh4, int m, int ny, const float2* twN, float2* A,
                               const float2* tw) {
    switch (nx) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        k4_rows_fwd<N><<<grid, L1Rows<N>::NT, L1Rows<N>::SMEM, s>>>(G, npairs, hh4, m, ny, twN, A, tw); \
        break;
        PCE_L1_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_l1_cols_inv(int ny, dim3 grid, cudaStream_t s, const float2* A, int nx, float* y,
                               float scale, const float2* tw) {
    switch (ny) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        k4_cols_inv<N><<<grid, ColCfg<N>::NT, ColCfg<N>::SMEM, s>>>(A, nx, y, scale, tw);      \
        break;
        PCE_L1_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_l1_rows_adj(int nx, dim3 grid, cudaStream_t s, const float2* V, int npairs,
                               const float2* hh4, int m, int ny, const float2* twN, float2* Q,
                               const float2* tw) {
    switch (nx) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        k4_rows_adj<N><<<grid, L1Rows<N>::NT, L1Rows<N>::SMEM, s>>>(V, npairs, hh4, m, ny, twN, Q, tw); \
        break;
        PCE_L1_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_l1_cols_adj(int ny, dim3 grid, cudaStream_t s, const float2* Q, int npairs,
                               const float* w, int m, int nx, float* x, float scale, const float2* tw) {
    switch (ny) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        k4_cols_adj<N><<<grid, ColCfg<N>::NT, ColCfg<N>::SMEM, s>>>(Q, npairs, w, m, nx, x, scale, tw); \
        break;
        PCE_L1_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_l1_rows_spec(int nx, dim3 grid, cudaStream_t s, const float2* G, int npairs, int m,
                                int ny, float2* hh4, const float2* tw) {
    switch (nx) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        k4_rows_spec<N><<<grid, L1Rows<N>::NT, L1Rows<N>::SMEM, s>>>(G, npairs, m, ny, hh4, tw); \
        break;
        PCE_L1_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t prepare_kernels() {
    cudaError_t e = prepare_cols();
    if (e == cudaSuccess) e = prepare_l1();
    if (e == cudaSuccess) e = prepare_sec();
#define X(N)                                                                                   \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_fwd_1d<N, float, float2, 1>,                                \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg1d<N, 1>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_adj_1d<N, float, float2, 1>,                                \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg1d<N, 1>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_fwd_1d<N, __nv_bfloat16, __half2, 1>,                       \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg1d<N, 1>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_adj_1d<N, __nv_bfloat16, __half2, 1>,                       \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg1d<N, 1>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_fwd_1d<N, float, float2>,                                   \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg1d<N>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_adj_1d<N, float, float2>,                                   \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg1d<N>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_fwd_1d<N, __nv_bfloat16, __half2>,                          \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg1d<N>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_adj_1d<N, __nv_bfloat16, __half2>,                          \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg1d<N>::SMEM); \
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

// Wide CTAs (more slots per right-hand side) when the batch leaves most SMs
// idle and the terms need more than one round of the narrow CTA's slots.
template <int N>
bool wide_1d(int batch, int m) {
    const int npairs = (m + 1) / 2;
    return Cfg1d<N, 1>::G > Cfg1d<N>::G && npairs > Cfg1d<N>::G && batch < 2 * 152;
}

// N = 1024 with few right-hand sides: the one-warp kernels (wk1d.cuh)
bool warp_1d(int n, int batch, const float2* tw1024) { return n == kWarpN && tw1024 && batch < 2 * 152; }

cudaError_t launch_fwd_1d(int n, int batch, cudaStream_t s, const float* u, const void* w,
                          const void* hp, const float* hscale, bool lowp, int m, float* y, float scale,
                          const float2* tw, const float2* tw1024) {
    using bf16 = __nv_bfloat16;
    if (warp_1d(n, batch, tw1024)) {
        if (lowp)
            kw_fwd_1d<bf16, __half2><<<batch, kW1dWarps * 32, 0, s>>>(
                u, static_cast<const bf16*>(w), static_cast<const __half2*>(hp), hscale, m, y, scale, tw1024);
        else
            kw_fwd_1d<float, float2><<<batch, kW1dWarps * 32, 0, s>>>(
                u, static_cast<const float*>(w), static_cast<const float2*>(hp), hscale, m, y, scale, tw1024);
        return cudaGetLastError();
    }
    switch (n) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        if (wide_1d<N>(batch, m)) {                                                            \
            if (lowp)                                                                          \
                k_fwd_1d<N, bf16, __half2, 1><<<batch, Cfg1d<N, 1>::NT, Cfg1d<N, 1>::SMEM, s>>>(  \
                    u, static_cast<const bf16*>(w), static_cast<const __half2*>(hp), hscale, m, y, \
                    scale, tw);                                                                \
            else                                                                               \
                k_fwd_1d<N, float, float2, 1><<<batch, Cfg1d<N, 1>::NT, Cfg1d<N, 1>::SMEM, s>>>(  \
                    u, static_cast<const float*>(w), static_cast<const float2*>(hp), hscale, m, y, \
                    scale, tw);                                                                \
        } else if (lowp)                                                                       \
            k_fwd_1d<N, bf16, __half2><<<batch, Cfg1d<N>::NT, Cfg1d<N>::SMEM, s>>>(              \
                u, static_cast<const bf16*>(w), static_cast<const __half2*>(hp), hscale, m, y,  \
                scale, tw);                                                                    \
        else                                                                                   \
            k_fwd_1d<N, float, float2><<<batch, Cfg1d<N>::NT, Cfg1d<N>::SMEM, s>>>(              \
                u, static_cast<const float*>(w), static_cast<const float2*>(hp), hscale, m, y,  \
                scale, tw);                                                                    \
        break;
        PCE_1D_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_1d(int n, int batch, cudaStream_t s, const float* v, const void* w,
                          const void* hp, const float* hscale, bool lowp, int m, float* x, float scale,
                          const float2* tw, const float2* tw1024) {
    using bf16 = __nv_bfloat16;
    if (warp_1d(n, batch, tw1024)) {
        if (lowp)
            kw_adj_1d<bf16, __half2><<<batch, kW1dWarps * 32, 0, s>>>(
                v, static_cast<const bf16*>(w), static_cast<const __half2*>(hp), hscale, m, x, scale, tw1024);
        else
            kw_adj_1d<float, float2><<<batch, kW1dWarps * 32, 0, s>>>(
                v, static_cast<const float*>(w), static_cast<const float2*>(hp), hscale, m, x, scale, tw1024);
        return cudaGetLastError();
    }
    switch (n) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        if (wide_1d<N>(batch, m)) {                                                            \
            if (lowp)                                                                          \
                k_adj_1d<N, bf16, __half2, 1><<<batch, Cfg1d<N, 1>::NT, Cfg1d<N, 1>::SMEM, s>>>(  \
                    v, static_cast<const bf16*>(w), static_cast<const __half2*>(hp), hscale, m, x, \
                    scale, tw);                                                                \
            else                                                                               \
                k_adj_1d<N, float, float2, 1><<<batch, Cfg1d<N, 1>::NT, Cfg1d<N, 1>::SMEM, s>>>(  \
                    v, static_cast<const float*>(w), static_cast<const float2*>(hp), hscale, m, x, \
                    scale, tw);                                                                \
        } else if (lowp)                                                                       \
            k_adj_1d<N, bf16, __half2><<<batch, Cfg1d<N>::NT, Cfg1d<N>::SMEM, s>>>(              \
                v, static_cast<const bf16*>(w), static_cast<const __half2*>(hp), hscale, m, x,  \
                scale, tw);                                                                    \
        else                                                                                   \
            k_adj_1d<N, float, float2><<<batch, Cfg1d<N>::NT, Cfg1d<N>::SMEM, s>>>(              \
                v, static_cast<const float*>(w), static_cast<const float2*>(hp), hscale, m, x,  \
                scale, tw);                                                                    \
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
