// wrows.cuh -- one-warp row kernels for the plain row transforms of rows of
// Nx = 1024 or 512 points: the R2C of the adjoint's input (G1) and the C2R of
// the forward's output (F3).
//
// They compute exactly what k_rows_r2c<NX, false> / k_rows_c2r<NX>
// (kernels.cuh) compute, with the same global layouts, but every row pair is
// transformed by one warp with the one-warp FFT of 1024 or 512 points (warpfft.cuh): one
// transpose through a warp-private shared tile and no CTA barrier per FFT,
// where the block Stockham kernels exchange through shared memory three times
// between CTA barriers.  Two real rows share one complex FFT, as in the block
// kernels.  (Windowed one-warp row passes -- the forward R2C with w_k and the
// adjoint's C2R-window-accumulate -- were measured slower than the block
// kernels, whose 48 resident warps per SM hide the extra window loads better
// than 16 one-warp FFTs can, and are not built.)
//
// Lane l reads the samples n = l + 32 q of both rows (coalesced 128-byte
// rows); after the forward FFT lane p holds Z[p + 32 m], and the half spectra
// of the two rows are separated with the partner Z[NX - f], read back from
// the warp's transpose tile.  The inverse direction loads the Hermitian
// extension of two packed half spectra (f >= NX / 2 read mirrored, still
// contiguous per warp) and stores x[p + 32 m] coalesced.
#pragma once

#include "wkernels.cuh"

namespace pce {

constexpr int kWRowWarps = 4;   // row pairs per CTA, one per warp

// the two rows' half spectra at f = lane + 32 m (m < NX / 64) from Z in v and
// the tile tr holding Z in natural order; slot 0 packs (X[0], X[NX / 2]) of
// each row
template <int NX>
__device__ __forceinline__ void wrow_split(const float2 (&v)[NX / 32], const float2* tr, int lane, int m, float2& A,
                                           float2& B) {
    const int f = lane + 32 * m;
    if (f == 0) {
        const float2 zn = tr[NX / 2];
        A = make_float2(v[0].x, zn.x);
        B = make_float2(v[0].y, zn.y);
    } else {
        const float2 z = v[m];
        const float2 zm = tr[NX - f];
        A = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
        B = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
    }
}

// G1: row pairs (2p, 2p + 1) of real rows -> their packed half spectra, one warp
// each; grid (ceil(npairs / 4), batch), 128 threads.
template <int NX>
__global__ void __launch_bounds__(kWRowWarps * 32)
kw_rows_r2c(const float* __restrict__ src, long long src_bstride, int nrows, float2* __restrict__ dst,
            long long dst_bstride, const float2* __restrict__ tw) {
    constexpr int NXh = NX / 2;
    constexpr int QN = NX / 32;
    __shared__ __align__(16) float2 trs[kWRowWarps][NX];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * kWRowWarps + warp;
    const int npairs = (nrows + 1) / 2;
    if (p >= npairs) return;   // warp-uniform; the kernel has no CTA barrier
    float2* tr = trs[warp];
    const int b = blockIdx.y;
    const RowItem<float> it = row_item<NX, false, float>(p, npairs, src + b * src_bstride, nrows, nullptr, nullptr,
                                                         nullptr);
    float2 v[QN];
#pragma unroll
    for (int q = 0; q < QN; ++q) {
        const int n = lane + 32 * q;
        v[q] = make_float2(it.va ? __ldg(it.sa + n) : 0.f, it.vb ? __ldg(it.sb + n) : 0.f);
    }
    warp_fft<NX, false>(v, tr, tw);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < QN; ++m) tr[lane + 32 * m] = v[m];
    __syncwarp();
    float2* da = dst + b * dst_bstride + (long long)it.la * NXh;
    float2* db = dst + b * dst_bstride + (long long)it.lb * NXh;
#pragma unroll
    for (int m = 0; m < QN / 2; ++m) {
        float2 A, B;
        wrow_split<NX>(v, tr, lane, m, A, B);
        if (it.va) da[lane + 32 * m] = A;
        if (it.vb) db[lane + 32 * m] = B;
    }
}

// the packed pair Za + i Zb of two rows' Hermitian-extended spectra at f = lane + 32 q
template <int NX>
__device__ __forceinline__ void wrow_load_pair(float2 (&v)[NX / 32], const float2* pa, const float2* pb, bool va,
                                               bool vb, int lane) {
#pragma unroll
    for (int q = 0; q < NX / 32; ++q) {
        const int f = lane + 32 * q;
        const float2 xa = va ? load_half<NX>(pa, f) : make_float2(0.f, 0.f);
        const float2 xb = vb ? load_half<NX>(pb, f) : make_float2(0.f, 0.f);
        v[q] = make_float2(xa.x - xb.y, xa.y + xb.x);
    }
}

// F3: rows pairs (2p, 2p + 1) of packed half spectra -> real rows times scale;
// grid (ceil(npairs / 4), batch), 128 threads.
template <int NX>
__global__ void __launch_bounds__(kWRowWarps * 32)
kw_rows_c2r(const float2* __restrict__ src, long long src_bstride, int nrows, float* __restrict__ dst,
            long long dst_bstride, float scale, const float2* __restrict__ tw) {
    constexpr int NXh = NX / 2;
    constexpr int QN = NX / 32;
    __shared__ __align__(16) float2 trs[kWRowWarps][NX];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * kWRowWarps + warp;
    const int npairs = (nrows + 1) / 2;
    if (p >= npairs) return;
    float2* tr = trs[warp];
    const int b = blockIdx.y;
    const int ga = 2 * p, gb = ga + 1;
    const bool vb = gb < nrows;
    const float2* pa = src + b * src_bstride + (long long)ga * NXh;
    const float2* pb = src + b * src_bstride + (long long)(vb ? gb : ga) * NXh;
    float2 v[QN];
    wrow_load_pair<NX>(v, pa, pb, true, vb, lane);
    warp_fft<NX, true>(v, tr, tw);
    float* xa = dst + b * dst_bstride + (long long)ga * NX;
    float* xb = dst + b * dst_bstride + (long long)gb * NX;
#pragma unroll
    for (int m = 0; m < QN; ++m) {
        xa[lane + 32 * m] = v[m].x * scale;
        if (vb) xb[lane + 32 * m] = v[m].y * scale;
    }
}

}  // namespace pce
