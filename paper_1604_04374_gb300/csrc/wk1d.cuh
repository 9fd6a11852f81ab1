// wk1d.cuh -- one-warp 1D applies for N = 1024 (few right-hand sides).
//
// The same operators as k_fwd_1d / k_adj_1d (kernels.cuh), with the same
// packed spectra, for the latency-bound case of a handful of right-hand
// sides: one CTA per right-hand side, whose warps take the term pairs in
// turn and run their FFTs with the one-warp 1024-point FFT (warpfft.cuh), so
// that no CTA barrier sits inside an FFT; the warps' partial sums meet once in
// shared memory at the end.  Lane l holds samples l + 32 q, and after a
// forward FFT frequencies l + 32 q (the four-step layout), so the products
// with the spectra and the windows are lane-local.
#pragma once

#include "wkernels.cuh"

namespace pce {

constexpr int kW1dWarps = 4;   // warps per CTA: term pairs in flight

// y_b = (1/N) C2R( sum_k hhat_k . R2C(w_k . u_b) ), N = 1024.  Grid (batch),
// kW1dWarps * 32 threads.  Warp w takes the term pairs w, w + kW1dWarps, ...:
// w_k u + i w_{k+1} u in one complex FFT, the two half spectra separated with
// the partner frequencies X[N - f] (shuffles), hhat . X accumulated for
// f = lane + 32 j (j < 16; lane 0, j = 0 packs the real DC and Nyquist terms
// as the packed spectra do).  Warp 0 sums the warps' half spectra and runs the
// inverse on their Hermitian extension.
template <typename WT, typename HT>
__global__ void __launch_bounds__(kW1dWarps * 32)
kw_fwd_1d(const float* __restrict__ u, const WT* __restrict__ w, const HT* __restrict__ hp,
          const float* __restrict__ hscale, int m, float* __restrict__ y, float scale,
          const float2* __restrict__ tw) {
    constexpr int N = kWarpN, Nh = N / 2;
    __shared__ __align__(16) float2 tiles[kW1dWarps][N];
    __shared__ __align__(16) float2 hsum[Nh];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* tr = tiles[warp];
    const int b = blockIdx.x;
    // the twiddles and the spectra are read after the first FFT's start and end
    prefetch_l2_block(tw, (long long)kWarpTwLen * sizeof(float2));
    prefetch_l2_block(hp, (long long)m * Nh * sizeof(HT));
    const float* ub = u + (long long)b * N;
    float ureg[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) ureg[q] = __ldg(ub + lane + 32 * q);
    float2 acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = make_float2(0.f, 0.f);
    const int npairs = (m + 1) / 2;
    for (int pr = warp; pr < npairs; pr += kW1dWarps) {
        const int k0 = 2 * pr, k1 = k0 + 1;
        const bool a1 = k1 < m;
        const WT* w0 = w + (long long)k0 * N;
        const WT* w1 = w + (long long)(a1 ? k1 : k0) * N;
        float2 v[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int n = lane + 32 * q;
            v[q] = make_float2(ldw(w0 + n) * ureg[q], a1 ? ldw(w1 + n) * ureg[q] : 0.f);
        }
        warp_fft1024<false>(v, tr, tw);
        const HT* h0 = hp + (long long)k0 * Nh;
        const HT* h1 = hp + (long long)(a1 ? k1 : k0) * Nh;
        const float s0 = hscale_of<HT>(hscale, k0);
        const float s1 = hscale_of<HT>(hscale, a1 ? k1 : k0);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int f = lane + 32 * j;
            const float2 zm = warp_partner(v, lane, j);   // every lane shuffles
            if (f == 0) {
                // real DC and Nyquist values of both terms: X0[0] = Z[0].x, X1[0] = Z[0].y,
                // X0[N/2] = Z[N/2].x, X1[N/2] = Z[N/2].y (Z[N/2] is lane 0's v[16])
                const float2 p0 = ldh(&h0[0], s0);
                acc[0].x = fmaf(p0.x, v[0].x, acc[0].x);
                acc[0].y = fmaf(p0.y, v[16].x, acc[0].y);
                if (a1) {
                    const float2 p1 = ldh(&h1[0], s1);
                    acc[0].x = fmaf(p1.x, v[0].y, acc[0].x);
                    acc[0].y = fmaf(p1.y, v[16].y, acc[0].y);
                }
            } else {
                float2 A, B;
                split_dc_nyq(v[j], zm, A, B);
                acc[j] = cfma(ldh(&h0[f], s0), A, acc[j]);
                if (a1) acc[j] = cfma(ldh(&h1[f], s1), B, acc[j]);
            }
        }
    }
    // the warps' half spectra, summed in warp order by warp 0
    __syncthreads();   // every warp is done with its transpose tile
#pragma unroll
    for (int j = 0; j < 16; ++j) tr[lane + 32 * j] = acc[j];
    __syncthreads();
    if (warp != 0) return;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        float2 s = tiles[0][lane + 32 * j];
        for (int g = 1; g < kW1dWarps; ++g) s = cadd(s, tiles[g][lane + 32 * j]);
        hsum[lane + 32 * j] = s;
    }
    __syncwarp();
    float2 v[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = load_half<N>(hsum, lane + 32 * q);
    warp_fft1024<true>(v, tr, tw);
    float* yb = y + (long long)b * N;
#pragma unroll
    for (int q = 0; q < 32; ++q) yb[lane + 32 * q] = v[q].x * scale;
}

// x_b = (1/N) sum_k w_k . IFFT( conj(hhat_k) . FFT(v_b) ), N = 1024.  Grid
// (batch), kW1dWarps * 32 threads.  Every warp transforms v itself, then takes
// the term pairs w, w + kW1dWarps, ...: the two inverse FFTs of a pair are
// real, so they share one complex inverse FFT; the windowed sums of the warps
// are added in warp order at the end.
template <typename WT, typename HT>
__global__ void __launch_bounds__(kW1dWarps * 32)
kw_adj_1d(const float* __restrict__ vin, const WT* __restrict__ w, const HT* __restrict__ hp,
          const float* __restrict__ hscale, int m, float* __restrict__ x, float scale,
          const float2* __restrict__ tw) {
    constexpr int N = kWarpN, Nh = N / 2;
    __shared__ __align__(16) float2 tiles[kW1dWarps][N];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* tr = tiles[warp];
    const int b = blockIdx.x;
    prefetch_l2_block(tw, (long long)kWarpTwLen * sizeof(float2));
    prefetch_l2_block(hp, (long long)m * Nh * sizeof(HT));
    prefetch_l2_block(w, (long long)m * N * sizeof(WT));
    const float* vb = vin + (long long)b * N;
    float2 V[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) V[q] = make_float2(__ldg(vb + lane + 32 * q), 0.f);
    warp_fft1024<false>(V, tr, tw);
    float ax[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) ax[q] = 0.f;
    const int npairs = (m + 1) / 2;
    for (int pr = warp; pr < npairs; pr += kW1dWarps) {
        const int k0 = 2 * pr, k1 = k0 + 1;
        const bool a1 = k1 < m;
        const HT* h0 = hp + (long long)k0 * Nh;
        const HT* h1 = hp + (long long)(a1 ? k1 : k0) * Nh;
        const float s0 = hscale_of<HT>(hscale, k0);
        const float s1 = hscale_of<HT>(hscale, a1 ? k1 : k0);
        float2 p[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int f = lane + 32 * q;
            float2 t = cmulc(V[q], load_half_h<N, HT>(h0, f, s0));
            if (a1) {
                const float2 s = cmulc(V[q], load_half_h<N, HT>(h1, f, s1));
                t.x -= s.y;
                t.y += s.x;
            }
            p[q] = t;
        }
        warp_fft1024<true>(p, tr, tw);
        const WT* w0 = w + (long long)k0 * N;
        const WT* w1 = w + (long long)(a1 ? k1 : k0) * N;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int n = lane + 32 * q;
            ax[q] = fmaf(ldw(w0 + n), p[q].x, ax[q]);
            if (a1) ax[q] = fmaf(ldw(w1 + n), p[q].y, ax[q]);
        }
    }
    __syncthreads();   // every warp is done with its transpose tile
    float* fb = reinterpret_cast<float*>(tr);
#pragma unroll
    for (int q = 0; q < 32; ++q) fb[lane + 32 * q] = ax[q];
    __syncthreads();
    if (warp != 0) return;
    float* xb = x + (long long)b * N;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        float s = reinterpret_cast<const float*>(tiles[0])[lane + 32 * q];
        for (int g = 1; g < kW1dWarps; ++g) s += reinterpret_cast<const float*>(tiles[g])[lane + 32 * q];
        xb[lane + 32 * q] = s * scale;
    }
}

}  // namespace pce
