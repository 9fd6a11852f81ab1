// cols.cu -- instances of the column-pass kernels for NY = 16 .. 2048 (one-warp
// kernels for NY = 512, 1024 and, two warps per column, 2048).
#include "kernels.cuh"
#include "wkernels.cuh"
#include "wkernels2.cuh"
#include "tkernels.cuh"
#include "launch.h"

namespace pce {

#define PCE_COL_SIZES(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048)

int cols_threads(int ny) {
    switch (ny) {
#define X(N) case N: return ColCfg<N>::NT;
        PCE_COL_SIZES(X)
#undef X
    }
    return 0;
}
int cols_columns_per_cta(int ny) {
    switch (ny) {
#define X(N) case N: return ColCfg<N>::C;
        PCE_COL_SIZES(X)
#undef X
    }
    return 0;
}
int cols_smem(int ny) {
    switch (ny) {
#define X(N) case N: return ColCfg<N>::SMEM;
        PCE_COL_SIZES(X)
#undef X
    }
    return 0;
}

cudaError_t prepare_cols() {
    cudaError_t e = cudaFuncSetAttribute(kw_cols_fwd<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWColSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kt_cols_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTColSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kt_cols_adj<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTColSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kt_cols_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTColSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kt_cols_adj<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTColSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kw2_cols_fwd<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kW2Smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kw2_cols_fwd<__half2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kW2Smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kw2_cols_adj<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kW2Smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kw2_cols_adj<__half2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kW2Smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kw_cols_fwd<__half2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWColSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kw_cols_adj<false, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kWColSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kw_cols_adj<false, __half2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kWColSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kw_cols_fwd<float2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kWColSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kw_cols_adj<false, float2, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kWColSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kw_cols_adj<true, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kWColSmem);
#define X(N)                                                                                   \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_cols_fwd<N, float2>,                                        \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<N>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_cols_fwd<N, __half2>,                                       \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<N>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_cols_adj<N, false, float2>,                                 \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<N>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_cols_adj<N, false, __half2>,                                \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<N>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_cols_adj<N, true, float2>,                                  \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<N>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_cols_grad_h<N>,                                             \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<N>::SMEM); \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_cols_spec<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                 ColCfg<N>::SMEM);                                             \
    if (e == cudaSuccess)                                                                      \
        e = cudaFuncSetAttribute(k_plain_cols_inv<N>,                                          \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<N>::SMEM);
    PCE_COL_SIZES(X)
#undef X
    return e;
}

cudaError_t launch_cols_fwd(int ny, dim3 grid, cudaStream_t s, const float2* Z, long long z_bstride,
                            long long z_kstride, const void* hh, const void* hN, const float* hscale,
                            bool lowp, int m,
                            const Box* box, int nxh, float2* A, long long a_bstride,
                            const float2* tw, const void* hhT, const float2* tw1024, int* status,
                            long long wait_limit, int skip_copy, bool warp,
                            const void* hN2, const float2* tw2048l) {
    // the warp-FFT column kernels index these tables: refuse to launch without them
    if ((ny == 512 || ny == kWarpN || ny == kW2N) && warp && (!tw1024 || !hhT)) return cudaErrorInvalidValue;
    if (ny == kW2N && warp && (!tw2048l || !hN2)) return cudaErrorInvalidValue;
    if (ny == kW2N && warp) {
        dim3 g2 = grid;
        if (lowp)
            kw2_cols_fwd<__half2><<<g2, 128, kW2Smem, s>>>(
                Z, z_bstride, z_kstride, static_cast<const __half2*>(hhT), static_cast<const __half2*>(hN2),
                hscale, m, box, nxh, A, a_bstride, tw1024, tw2048l, status, wait_limit, skip_copy);
        else
            kw2_cols_fwd<float2><<<g2, 128, kW2Smem, s>>>(
                Z, z_bstride, z_kstride, static_cast<const float2*>(hhT), static_cast<const float2*>(hN2),
                hscale, m, box, nxh, A, a_bstride, tw1024, tw2048l, status, wait_limit, skip_copy);
        return cudaGetLastError();
    }
    if (ny == kWarpN && warp) {
        if (lowp)
            kw_cols_fwd<__half2><<<grid, kWColWarps * 32, kWColSmem, s>>>(
                Z, z_bstride, z_kstride, static_cast<const __half2*>(hhT), static_cast<const __half2*>(hN),
                hscale, m, box, nxh, A, a_bstride, tw1024, status, wait_limit, skip_copy);
        else
            kw_cols_fwd<float2><<<grid, kWColWarps * 32, kWColSmem, s>>>(
                Z, z_bstride, z_kstride, static_cast<const float2*>(hhT), static_cast<const float2*>(hN),
                hscale, m, box, nxh, A, a_bstride, tw1024, status, wait_limit, skip_copy);
        return cudaGetLastError();
    }
    if (ny == 512 && warp) {
        constexpr int sm = kw_col_smem<512>();
        if (lowp)
            kw_cols_fwd<__half2, false, 512><<<grid, kWColWarps * 32, sm, s>>>(
                Z, z_bstride, z_kstride, static_cast<const __half2*>(hhT), static_cast<const __half2*>(hN),
                hscale, m, box, nxh, A, a_bstride, tw1024, status, wait_limit, skip_copy);
        else
            kw_cols_fwd<float2, false, 512><<<grid, kWColWarps * 32, sm, s>>>(
                Z, z_bstride, z_kstride, static_cast<const float2*>(hhT), static_cast<const float2*>(hN),
                hscale, m, box, nxh, A, a_bstride, tw1024, status, wait_limit, skip_copy);
        return cudaGetLastError();
    }
    switch (ny) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        if (lowp)                                                                              \
            k_cols_fwd<N, __half2><<<grid, ColCfg<N>::NT, ColCfg<N>::SMEM, s>>>(                 \
                Z, z_bstride, z_kstride, static_cast<const __half2*>(hh),                      \
                static_cast<const __half2*>(hN), hscale, m, box, nxh, A, a_bstride, tw);        \
        else                                                                                   \
            k_cols_fwd<N, float2><<<grid, ColCfg<N>::NT, ColCfg<N>::SMEM, s>>>(                  \
                Z, z_bstride, z_kstride, static_cast<const float2*>(hh),                       \
                static_cast<const float2*>(hN), hscale, m, box, nxh, A, a_bstride, tw);         \
        break;
        PCE_COL_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_cols_adj(int ny, dim3 grid, cudaStream_t s, const float2* V, long long v_bstride,
                            const void* hh, const void* hN, const float* hscale, bool lowp, int m,
                            const Box* box, int nxh, float2* Q, long long q_bstride, long long q_kstride,
                            const float2* tw, const void* hhT, const float2* tw1024, int* status,
                            long long wait_limit, int skip_copy, bool warp,
                            const void* hN2, const float2* tw2048l) {
    if ((ny == 512 || ny == kWarpN || ny == kW2N) && warp && (!tw1024 || !hhT)) return cudaErrorInvalidValue;
    if (ny == kW2N && warp && (!tw2048l || !hN2)) return cudaErrorInvalidValue;
    if (ny == kW2N && warp) {
        if (lowp)
            kw2_cols_adj<__half2><<<grid, 128, kW2Smem, s>>>(
                V, v_bstride, static_cast<const __half2*>(hhT), static_cast<const __half2*>(hN2), hscale, m,
                box, nxh, Q, q_bstride, q_kstride, tw1024, tw2048l, status, wait_limit, skip_copy);
        else
            kw2_cols_adj<float2><<<grid, 128, kW2Smem, s>>>(
                V, v_bstride, static_cast<const float2*>(hhT), static_cast<const float2*>(hN2), hscale, m,
                box, nxh, Q, q_bstride, q_kstride, tw1024, tw2048l, status, wait_limit, skip_copy);
        return cudaGetLastError();
    }
    if (ny == kWarpN && warp) {
        if (lowp)
            kw_cols_adj<false, __half2><<<grid, kWColWarps * 32, kWColSmem, s>>>(
                V, v_bstride, static_cast<const __half2*>(hhT), static_cast<const __half2*>(hN), hscale, m,
                box, nxh, Q, q_bstride, q_kstride, tw1024, status, wait_limit, skip_copy);
        else
            kw_cols_adj<false, float2><<<grid, kWColWarps * 32, kWColSmem, s>>>(
                V, v_bstride, static_cast<const float2*>(hhT), static_cast<const float2*>(hN), hscale, m,
                box, nxh, Q, q_bstride, q_kstride, tw1024, status, wait_limit, skip_copy);
        return cudaGetLastError();
    }
    if (ny == 512 && warp) {
        constexpr int sm = kw_col_smem<512>();
        if (lowp)
            kw_cols_adj<false, __half2, false, 512><<<grid, kWColWarps * 32, sm, s>>>(
                V, v_bstride, static_cast<const __half2*>(hhT), static_cast<const __half2*>(hN), hscale, m,
                box, nxh, Q, q_bstride, q_kstride, tw1024, status, wait_limit, skip_copy);
        else
            kw_cols_adj<false, float2, false, 512><<<grid, kWColWarps * 32, sm, s>>>(
                V, v_bstride, static_cast<const float2*>(hhT), static_cast<const float2*>(hN), hscale, m,
                box, nxh, Q, q_bstride, q_kstride, tw1024, status, wait_limit, skip_copy);
        return cudaGetLastError();
    }
    switch (ny) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        if (lowp)                                                                              \
            k_cols_adj<N, false, __half2><<<grid, ColCfg<N>::NT, ColCfg<N>::SMEM, s>>>(          \
                V, v_bstride, static_cast<const __half2*>(hh), static_cast<const __half2*>(hN),  \
                hscale, m, box, nxh, Q, q_bstride, q_kstride, tw);                             \
        else                                                                                   \
            k_cols_adj<N, false, float2><<<grid, ColCfg<N>::NT, ColCfg<N>::SMEM, s>>>(           \
                V, v_bstride, static_cast<const float2*>(hh), static_cast<const float2*>(hN),    \
                hscale, m, box, nxh, Q, q_bstride, q_kstride, tw);                             \
        break;
        PCE_COL_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_cols_spec(int ny, dim3 grid, cudaStream_t s, const float2* S, int nxh,
                             float2* hh, float2* hN, const float2* tw) {
    switch (ny) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        k_cols_spec<N><<<grid, ColCfg<N>::NT, ColCfg<N>::SMEM, s>>>(S, nxh, hh, hN, tw);        \
        break;
        PCE_COL_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_plain_cols_inv(int ny, dim3 grid, cudaStream_t s, const float2* acc,
                                  const float2* accN, int nxh, float2* A, const float2* tw) {
    switch (ny) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        k_plain_cols_inv<N><<<grid, ColCfg<N>::NT, ColCfg<N>::SMEM, s>>>(acc, accN, nxh, A, tw); \
        break;
        PCE_COL_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_cols_fwd_sep(int ny, dim3 grid, cudaStream_t s, const float2* Z, long long z_bstride,
                                long long z_kstride, const float2* hhT, const float2* hN, int m,
                                const Box* box, int nxh, float2* A, long long a_bstride,
                                const float2* tw1024, int* status, long long wait_limit, int skip_copy,
                                const SepTerms& sep) {
    if (!tw1024 || !hhT) return cudaErrorInvalidValue;
    if (ny == kWarpN)
        kw_cols_fwd<float2, true><<<grid, kWColWarps * 32, kWColSmem, s>>>(
            Z, z_bstride, z_kstride, hhT, hN, nullptr, m, box, nxh, A, a_bstride, tw1024, status, wait_limit,
            skip_copy, sep);
    else if (ny == 512)
        kw_cols_fwd<float2, true, 512><<<grid, kWColWarps * 32, kw_col_smem<512>(), s>>>(
            Z, z_bstride, z_kstride, hhT, hN, nullptr, m, box, nxh, A, a_bstride, tw1024, status, wait_limit,
            skip_copy, sep);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_cols_adj_sep(int ny, dim3 grid, cudaStream_t s, const float2* V, long long v_bstride,
                                const float2* hhT, const float2* hN, int m, const Box* box, int nxh,
                                float2* Q, long long q_bstride, long long q_kstride,
                                const float2* tw1024, int* status, long long wait_limit, int skip_copy,
                                const SepTerms& sep) {
    if (!tw1024 || !hhT) return cudaErrorInvalidValue;
    if (ny == kWarpN)
        kw_cols_adj<false, float2, true><<<grid, kWColWarps * 32, kWColSmem, s>>>(
            V, v_bstride, hhT, hN, nullptr, m, box, nxh, Q, q_bstride, q_kstride, tw1024, status, wait_limit,
            skip_copy, sep);
    else if (ny == 512)
        kw_cols_adj<false, float2, true, 512><<<grid, kWColWarps * 32, kw_col_smem<512>(), s>>>(
            V, v_bstride, hhT, hN, nullptr, m, box, nxh, Q, q_bstride, q_kstride, tw1024, status, wait_limit,
            skip_copy, sep);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_cols_fwd_sep_tm(int ny, dim3 grid, cudaStream_t s, const float2* Z, long long z_bstride,
                                   long long z_kstride, const float2* hhT, const float2* hN, const Box* box,
                                   int nxh, float2* A, long long a_bstride, const float2* tw1024, int* status,
                                   long long wait_limit, int skip_copy, const SepTerms& sep) {
    if (!tw1024 || !hhT) return cudaErrorInvalidValue;
    if (ny == 512 && !sep.kq0) {   // 512-point columns: no pruned form
        kt_cols_fwd<false, 512><<<grid, kWColWarps * 32, kt_smem<512>(), s>>>(
            Z, z_bstride, z_kstride, hhT, hN, box, nxh, A, a_bstride, tw1024, status, wait_limit, skip_copy, sep);
        return cudaGetLastError();
    }
    if (ny != kWarpN) return cudaErrorInvalidValue;
    if (sep.kq0)
        kt_cols_fwd<true><<<grid, kWColWarps * 32, kTColSmem, s>>>(Z, z_bstride, z_kstride, hhT, hN, box, nxh, A,
                                                                   a_bstride, tw1024, status, wait_limit, skip_copy,
                                                                   sep);
    else
        kt_cols_fwd<false><<<grid, kWColWarps * 32, kTColSmem, s>>>(Z, z_bstride, z_kstride, hhT, hN, box, nxh, A,
                                                                    a_bstride, tw1024, status, wait_limit,
                                                                    skip_copy, sep);
    return cudaGetLastError();
}

cudaError_t launch_cols_adj_sep_tm(int ny, dim3 grid, cudaStream_t s, float2* V, long long v_bstride,
                                   const float2* hhT, const float2* hN, const Box* box, int nxh, float2* Q,
                                   long long q_bstride, long long q_kstride, const float2* tw1024, int* status,
                                   long long wait_limit, int skip_copy, const SepTerms& sep) {
    if (!tw1024 || !hhT) return cudaErrorInvalidValue;
    if (ny == 512 && !sep.kq0) {
        kt_cols_adj<false, 512><<<grid, kWColWarps * 32, kt_smem<512>(), s>>>(
            V, v_bstride, hhT, hN, box, nxh, Q, q_bstride, q_kstride, tw1024, status, wait_limit, skip_copy, sep);
        return cudaGetLastError();
    }
    if (ny != kWarpN) return cudaErrorInvalidValue;
    if (sep.kq0)
        kt_cols_adj<true><<<grid, kWColWarps * 32, kTColSmem, s>>>(V, v_bstride, hhT, hN, box, nxh, Q, q_bstride,
                                                                   q_kstride, tw1024, status, wait_limit, skip_copy,
                                                                   sep);
    else
        kt_cols_adj<false><<<grid, kWColWarps * 32, kTColSmem, s>>>(V, v_bstride, hhT, hN, box, nxh, Q, q_bstride,
                                                                    q_kstride, tw1024, status, wait_limit,
                                                                    skip_copy, sep);
    return cudaGetLastError();
}

cudaError_t launch_cols_adj_full(int ny, dim3 grid, cudaStream_t s, const float2* V, long long v_bstride,
                                 const float2* hh, const float2* hN, int m, const Box* box, int nxh,
                                 float2* Q, long long q_bstride, long long q_kstride,
                                 const float2* tw, const float2* hhT, const float2* tw1024, int* status,
                                 long long wait_limit, int skip_copy) {
    if (ny == kWarpN) {
        kw_cols_adj<true, float2><<<grid, kWColWarps * 32, kWColSmem, s>>>(
            V, v_bstride, hhT, hN, nullptr, m, box, nxh, Q, q_bstride, q_kstride, tw1024, status, wait_limit,
            skip_copy);
        return cudaGetLastError();
    }
    if (ny == 512 && hhT && tw1024) {
        kw_cols_adj<true, float2, false, 512><<<grid, kWColWarps * 32, kw_col_smem<512>(), s>>>(
            V, v_bstride, hhT, hN, nullptr, m, box, nxh, Q, q_bstride, q_kstride, tw1024, status, wait_limit,
            skip_copy);
        return cudaGetLastError();
    }
    switch (ny) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        k_cols_adj<N, true, float2><<<grid, ColCfg<N>::NT, ColCfg<N>::SMEM, s>>>(                \
            V, v_bstride, hh, hN, nullptr, m, box, nxh, Q, q_bstride, q_kstride, tw);         \
        break;
        PCE_COL_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_cols_grad_h(int ny, dim3 grid, cudaStream_t s, const float2* Z, long long z_bstride,
                               long long z_kstride, int nb, const float2* Rh, const float2* RhN,
                               const Box* box, int nxh, float2* dhh, float scale, int accumulate,
                               const float2* tw) {
    switch (ny) {
#define X(N)                                                                                   \
    case N:                                                                                    \
        k_cols_grad_h<N><<<grid, ColCfg<N>::NT, ColCfg<N>::SMEM, s>>>(                          \
            Z, z_bstride, z_kstride, nb, Rh, RhN, box, nxh, dhh, scale, accumulate, tw);       \
        break;
        PCE_COL_SIZES(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pce
