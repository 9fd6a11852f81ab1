// sect.cu -- instances and launchers of the sectioned-apply kernels.
#include "section.cuh"
#include "launch.h"

namespace pce {

// the host sizes the sectioned column grid with cols_columns_per_cta(1024)
static_assert(ColCfg<1024>::C == kWColWarps, "columns per CTA of the 1024-point column kernels");

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
    const void* fns[] = {(const void*)kw_sec_cols<false, float2>, (const void*)kw_sec_cols<true, float2>,
                         (const void*)kw_sec_cols<false, __half2>, (const void*)kw_sec_cols<true, __half2>};
    for (const void* f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kSecColSmem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {

template <int N, typename WT>
void sec_r2c(bool win, dim3 grid, cudaStream_t s, const float* src, long long src_bstride, int nyg, int nxg,
             const WT* wbox, const SecGeom* geo, const int2* items, int nitems, float2* dst, long long dst_bstride,
             long long dst_kstride, const float2* tw) {
    if (win)
        k_sec_r2c<N, true, WT><<<grid, 256, 0, s>>>(src, src_bstride, nyg, nxg, wbox, geo, items, nitems, dst,
                                                    dst_bstride, dst_kstride, tw);
    else
        k_sec_r2c<N, false, WT><<<grid, 256, 0, s>>>(src, src_bstride, nyg, nxg, wbox, geo, items, nitems, dst,
                                                     dst_bstride, dst_kstride, tw);
}

template <int N, typename WT>
void sec_c2r(bool win, dim3 grid, cudaStream_t s, const float2* src, long long src_bstride, long long src_kstride,
             const SecGeom* geo, const int2* items, int nitems, const WT* wbox, float* dst, long long dst_bstride,
             int nyg, int nxg, float scale, const float2* tw) {
    if (win)
        k_sec_c2r<N, true, WT><<<grid, 256, 0, s>>>(src, src_bstride, src_kstride, geo, items, nitems, wbox, dst,
                                                    dst_bstride, nyg, nxg, scale, tw);
    else
        k_sec_c2r<N, false, WT><<<grid, 256, 0, s>>>(src, src_bstride, src_kstride, geo, items, nitems, wbox, dst,
                                                     dst_bstride, nyg, nxg, scale, tw);
}

template <bool CONJ, typename HT>
void sec_cols(dim3 grid, cudaStream_t s, const float2* Z, long long z_bstride, long long z_kstride, int nb,
              const void* hsT, const void* hsN, const float* hscale, const SecGeom* geo, int nxh, float2* A,
              long long a_bstride, long long a_kstride, const float2* tw1024, int* status, long long wait_limit,
              int skip_copy) {
    kw_sec_cols<CONJ, HT><<<grid, kWColWarps * 32, kSecColSmem, s>>>(
        Z, z_bstride, z_kstride, nb, static_cast<const HT*>(hsT), static_cast<const HT*>(hsN), hscale, geo, nxh, A,
        a_bstride, a_kstride, tw1024, status, wait_limit, skip_copy);
}

}  // namespace

cudaError_t launch_sec_r2c(int lc, bool win, dim3 grid, cudaStream_t s, const float* src, long long src_bstride,
                           int nyg, int nxg, const void* wbox, bool lowp, const SecGeom* geo, const int2* items,
                           int nitems, float2* dst, long long dst_bstride, long long dst_kstride, const float2* tw) {
    switch (lc) {
#define X(N)                                                                                                   \
    case N:                                                                                                    \
        if (lowp)                                                                                              \
            sec_r2c<N>(win, grid, s, src, src_bstride, nyg, nxg, static_cast<const __nv_bfloat16*>(wbox), geo, \
                       items, nitems, dst, dst_bstride, dst_kstride, tw);                                      \
        else                                                                                                   \
            sec_r2c<N>(win, grid, s, src, src_bstride, nyg, nxg, static_cast<const float*>(wbox), geo, items,  \
                       nitems, dst, dst_bstride, dst_kstride, tw);                                             \
        break;
        PCE_SEC_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_sec_cols(bool conj, dim3 grid, cudaStream_t s, const float2* Z, long long z_bstride,
                            long long z_kstride, int nb, const void* hsT, const void* hsN, const float* hscale,
                            bool lowp, const SecGeom* geo, int nxh, float2* A, long long a_bstride,
                            long long a_kstride, const float2* tw1024, int* status, long long wait_limit,
                            int skip_copy) {
    if (!tw1024 || !hsT || !hsN || (lowp && !hscale)) return cudaErrorInvalidValue;
    if (lowp) {
        if (conj)
            sec_cols<true, __half2>(grid, s, Z, z_bstride, z_kstride, nb, hsT, hsN, hscale, geo, nxh, A, a_bstride,
                                    a_kstride, tw1024, status, wait_limit, skip_copy);
        else
            sec_cols<false, __half2>(grid, s, Z, z_bstride, z_kstride, nb, hsT, hsN, hscale, geo, nxh, A, a_bstride,
                                     a_kstride, tw1024, status, wait_limit, skip_copy);
    } else {
        if (conj)
            sec_cols<true, float2>(grid, s, Z, z_bstride, z_kstride, nb, hsT, hsN, hscale, geo, nxh, A, a_bstride,
                                   a_kstride, tw1024, status, wait_limit, skip_copy);
        else
            sec_cols<false, float2>(grid, s, Z, z_bstride, z_kstride, nb, hsT, hsN, hscale, geo, nxh, A, a_bstride,
                                    a_kstride, tw1024, status, wait_limit, skip_copy);
    }
    return cudaGetLastError();
}

cudaError_t launch_sec_c2r(int lc, bool win, dim3 grid, cudaStream_t s, const float2* src, long long src_bstride,
                           long long src_kstride, const SecGeom* geo, const int2* items, int nitems,
                           const void* wbox, bool lowp, float* dst, long long dst_bstride, int nyg, int nxg,
                           float scale, const float2* tw) {
    switch (lc) {
#define X(N)                                                                                                   \
    case N:                                                                                                    \
        if (lowp)                                                                                              \
            sec_c2r<N>(win, grid, s, src, src_bstride, src_kstride, geo, items, nitems,                        \
                       static_cast<const __nv_bfloat16*>(wbox), dst, dst_bstride, nyg, nxg, scale, tw);        \
        else                                                                                                   \
            sec_c2r<N>(win, grid, s, src, src_bstride, src_kstride, geo, items, nitems,                        \
                       static_cast<const float*>(wbox), dst, dst_bstride, nyg, nxg, scale, tw);                \
        break;
        PCE_SEC_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pce
