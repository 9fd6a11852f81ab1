// sect.cu -- instances and launchers of the sectioned-apply kernels.
#include "section.cuh"
#include "launch.h"

namespace pce {

#define PCE_SEC_SIZES(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048)

int sec_rows_per_cta(int lc) {
    switch (lc) {
#define X(N) case N: return 256 / (N / kR) > 0 ? 256 / (N / kR) : 1;
        PCE_SEC_SIZES(X)
#undef X
    }
    return 0;
}

cudaError_t prepare_sec() {
    cudaError_t e = cudaFuncSetAttribute(kw_sec_cols<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWColSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kw_sec_cols<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWColSmem);
    return e;
}

cudaError_t launch_sec_r2c(int lc, bool win, dim3 grid, cudaStream_t s, const float* src, long long src_bstride,
                           int nyg, int nxg, const float* wbox, const SecGeom* geo, const int2* items, int nitems,
                           float2* dst, long long dst_bstride, long long dst_kstride, const float2* tw) {
    switch (lc) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        if (win)                                                                               \
            k_sec_r2c<N, true><<<grid, 256, 0, s>>>(src, src_bstride, nyg, nxg, wbox, geo, items, nitems, \
                                                    dst, dst_bstride, dst_kstride, tw);        \
        else                                                                                   \
            k_sec_r2c<N, false><<<grid, 256, 0, s>>>(src, src_bstride, nyg, nxg, wbox, geo, items, nitems, \
                                                     dst, dst_bstride, dst_kstride, tw);       \
        break;
        PCE_SEC_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_sec_cols(bool conj, dim3 grid, cudaStream_t s, const float2* Z, long long z_bstride,
                            long long z_kstride, int nb, const float2* hsT, const float2* hsN, const SecGeom* geo,
                            int nxh, float2* A, long long a_bstride, long long a_kstride, const float2* tw1024,
                            int* status, long long wait_limit, int skip_copy) {
    if (!tw1024 || !hsT || !hsN) return cudaErrorInvalidValue;
    if (conj)
        kw_sec_cols<true><<<grid, kWColWarps * 32, kWColSmem, s>>>(Z, z_bstride, z_kstride, nb, hsT, hsN, geo, nxh,
                                                                   A, a_bstride, a_kstride, tw1024, status, wait_limit, skip_copy);
    else
        kw_sec_cols<false><<<grid, kWColWarps * 32, kWColSmem, s>>>(Z, z_bstride, z_kstride, nb, hsT, hsN, geo, nxh,
                                                                    A, a_bstride, a_kstride, tw1024, status, wait_limit, skip_copy);
    return cudaGetLastError();
}

cudaError_t launch_sec_c2r(int lc, bool win, dim3 grid, cudaStream_t s, const float2* src, long long src_bstride,
                           long long src_kstride, const SecGeom* geo, const int2* items, int nitems,
                           const float* wbox, float* dst, long long dst_bstride, int nyg, int nxg, float scale,
                           const float2* tw) {
    switch (lc) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        if (win)                                                                               \
            k_sec_c2r<N, true><<<grid, 256, 0, s>>>(src, src_bstride, src_kstride, geo, items, nitems, wbox, \
                                                    dst, dst_bstride, nyg, nxg, scale, tw);    \
        else                                                                                   \
            k_sec_c2r<N, false><<<grid, 256, 0, s>>>(src, src_bstride, src_kstride, geo, items, nitems, wbox, \
                                                     dst, dst_bstride, nyg, nxg, scale, tw);   \
        break;
        PCE_SEC_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pce
