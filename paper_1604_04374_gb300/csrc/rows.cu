// rows.cu -- instances of the row-pass kernels for NX = 16 .. 2048.
#include "kernels.cuh"
#include "launch.h"
#include "wrows.cuh"

namespace pce {

int rows_pairs_per_cta(int nx) { return 256 / (nx / kR); }
int rows_grad_pairs_per_cta(int nx) { return 256 / (nx / kR); }
int rows_r2c_items_per_cta(int nx) { return kRowIters * (256 / (nx / kR)); }

#define PCE_ROW_SIZES(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048)

cudaError_t launch_rows_r2c(int nx, bool window, dim3 grid, cudaStream_t s,
                            const float* src, long long src_bstride, int nrows,
                            const void* wbox, bool lowp, const Box* box, const int2* items, int nitems,
                            float2* dst, long long dst_bstride, long long dst_kstride,
                            const float2* tw, const float2* /*tw1024*/) {
    using bf16 = __nv_bfloat16;
    switch (nx) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        if (window && lowp)                                                                    \
            k_rows_r2c<N, true, bf16><<<grid, 256, 0, s>>>(src, src_bstride, nrows,            \
                                                          static_cast<const bf16*>(wbox), box,  \
                                                          items, nitems, dst, dst_bstride,     \
                                                          dst_kstride, tw);                    \
        else if (window)                                                                       \
            k_rows_r2c<N, true, float><<<grid, 256, 0, s>>>(src, src_bstride, nrows,           \
                                                           static_cast<const float*>(wbox), box, \
                                                           items, nitems, dst, dst_bstride,    \
                                                           dst_kstride, tw);                   \
        else                                                                                   \
            k_rows_r2c<N, false, float><<<grid, 256, 0, s>>>(src, src_bstride, nrows, nullptr,  \
                                                            box, items, nitems, dst,           \
                                                            dst_bstride, dst_kstride, tw);     \
        break;
        PCE_ROW_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rows_r2c_pairs(int nx, int nb, cudaStream_t s, const float* src, long long src_bstride,
                                  int nrows, const void* wbox, bool lowp, const Box* box, const int* kptr,
                                  const int* klist, float2* dst, long long dst_bstride, long long dst_kstride,
                                  const float2* tw) {
    using bf16 = __nv_bfloat16;
    const int npairs = (nrows + 1) / 2;
    switch (nx) {
#define X(N)                                                                                      \
    case N: {                                                                                     \
        const int fpc = rows_pairs_per_cta(N);                                                    \
        const dim3 grid((npairs + fpc - 1) / fpc, nb);                                            \
        if (lowp)                                                                                 \
            k_rows_r2c_pairs<N, bf16><<<grid, 256, 0, s>>>(src, src_bstride, nrows,                \
                                                         static_cast<const bf16*>(wbox), box, kptr, \
                                                         klist, dst, dst_bstride, dst_kstride, tw); \
        else                                                                                      \
            k_rows_r2c_pairs<N, float><<<grid, 256, 0, s>>>(src, src_bstride, nrows,               \
                                                          static_cast<const float*>(wbox), box, kptr, \
                                                          klist, dst, dst_bstride, dst_kstride, tw); \
        break;                                                                                    \
    }
        PCE_ROW_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rows_c2r(int nx, dim3 grid, cudaStream_t s, const float2* src,
                            long long src_bstride, int nrows, float* dst, long long dst_bstride,
                            float scale, const float2* tw, const float2* /*tw1024*/) {
    switch (nx) {
#define X(N)                                                                                  \
    case N:                                                                                   \
        k_rows_c2r<N><<<grid, 256, 0, s>>>(src, src_bstride, nrows, dst, dst_bstride, scale, tw); \
        break;
        PCE_ROW_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rows_adj(int nx, dim3 grid, cudaStream_t s, const float2* Q, long long q_bstride,
                            long long q_kstride, int nrows, const void* wbox, bool lowp, const Box* box,
                            const int* kptr, const int* klist, float* dst, long long dst_bstride,
                            float scale, const float2* tw, const float2* /*tw1024*/, int rv, int kmin, int kmax,
                            int accumulate) {
    using bf16 = __nv_bfloat16;
    switch (nx) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        if (lowp && rv)                                                                        \
            k_rows_adj<N, bf16, 1><<<grid, 256, 0, s>>>(Q, q_bstride, q_kstride, nrows,         \
                                                       static_cast<const bf16*>(wbox), box,    \
                                                       kptr, klist, dst, dst_bstride, scale, tw, kmin, kmax, accumulate); \
        else if (lowp)                                                                         \
            k_rows_adj<N, bf16, 0><<<grid, 256, 0, s>>>(Q, q_bstride, q_kstride, nrows,         \
                                                       static_cast<const bf16*>(wbox), box,    \
                                                       kptr, klist, dst, dst_bstride, scale, tw, kmin, kmax, accumulate); \
        else if (rv)                                                                           \
            k_rows_adj<N, float, 1><<<grid, 256, 0, s>>>(Q, q_bstride, q_kstride, nrows,        \
                                                        static_cast<const float*>(wbox), box,  \
                                                        kptr, klist, dst, dst_bstride, scale, tw, kmin, kmax, accumulate); \
        else                                                                                   \
            k_rows_adj<N, float, 0><<<grid, 256, 0, s>>>(Q, q_bstride, q_kstride, nrows,        \
                                                        static_cast<const float*>(wbox), box,  \
                                                        kptr, klist, dst, dst_bstride, scale, tw, kmin, kmax, accumulate); \
        break;
        PCE_ROW_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_wrows_r2c(int nx, int nb, cudaStream_t s, const float* src, long long src_bstride, int nrows,
                             float2* dst, long long dst_bstride, const float2* tw1024) {
    if (!tw1024) return cudaErrorInvalidValue;
    const int npairs = (nrows + 1) / 2;
    const dim3 grid((npairs + kWRowWarps - 1) / kWRowWarps, nb);
    if (nx == kWarpN)
        kw_rows_r2c<kWarpN><<<grid, kWRowWarps * 32, 0, s>>>(src, src_bstride, nrows, dst, dst_bstride, tw1024);
    else if (nx == 512)
        kw_rows_r2c<512><<<grid, kWRowWarps * 32, 0, s>>>(src, src_bstride, nrows, dst, dst_bstride, tw1024);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_wrows_c2r(int nx, int nb, cudaStream_t s, const float2* src, long long src_bstride, int nrows,
                             float* dst, long long dst_bstride, float scale, const float2* tw1024) {
    if (!tw1024) return cudaErrorInvalidValue;
    const int npairs = (nrows + 1) / 2;
    const dim3 grid((npairs + kWRowWarps - 1) / kWRowWarps, nb);
    if (nx == kWarpN)
        kw_rows_c2r<kWarpN><<<grid, kWRowWarps * 32, 0, s>>>(src, src_bstride, nrows, dst, dst_bstride, scale,
                                                              tw1024);
    else if (nx == 512)
        kw_rows_c2r<512><<<grid, kWRowWarps * 32, 0, s>>>(src, src_bstride, nrows, dst, dst_bstride, scale, tw1024);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_rows_grad_w(int nx, dim3 grid, cudaStream_t s, const float2* Qf, long long q_bstride,
                               long long q_kstride, int nrows, int nb, const float* u,
                               long long u_bstride, float* dw, float scale, int accumulate,
                               const float2* tw) {
    switch (nx) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        k_rows_grad_w<N><<<grid, 256, 0, s>>>(Qf, q_bstride, q_kstride, nrows, nb, u, u_bstride, \
                                              dw, scale, accumulate, tw);                      \
        break;
        PCE_ROW_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pce
