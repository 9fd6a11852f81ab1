// wkernels2.cuh -- column kernels for columns of length Ny = 2048, two warps
// per column, each running the one-warp 1024-point FFT of warpfft.cuh.
//
// Decimation in frequency splits a 2048-point DFT into two 1024-point ones:
//   X[2k]     = DFT1024( x[n] + x[n+1024] )[k]
//   X[2k + 1] = DFT1024( (x[n] - x[n+1024]) W2048^n )[k]
// Warp `par` of a column (par = 0 even, 1 odd frequencies) forms its input
// from the two halves of the column, which both sit in the shared column
// tile, so the per-term loop needs no exchange between the two warps.  Each
// warp multiplies its half of the spectrum by the matching half of hhat_k
// (stored de-interleaved: [k][column][par][1024]).  The inverse runs the two
// halves backwards: a = IDFT1024(A_even), b' = W2048^{-n} IDFT1024(A_odd),
// x[n] = a + b', x[n+1024] = a - b' (unnormalised), combined while the
// column is staged in the tile for the store.
//
// CTA: 4 warps = 2 columns.  Shared memory: the column tile [2048][2]
// (column index XOR-swizzled by (row >> 3) & 1) and one 1024-point transpose
// tile per warp.  W2048^{l + 32 q} = W2048^l W64^q: one table value per lane
// and compile-time constants.
#pragma once

#include "wkernels.cuh"

namespace pce {

constexpr int kW2N = 2048;
constexpr int kW2Cols = 2;   // columns per CTA
constexpr int kW2Smem = (kW2N * kW2Cols + 4 * kWarpN) * (int)sizeof(float2);

__device__ __forceinline__ int tix2(int row, int c) { return 2 * row + (c ^ ((row >> 3) & 1)); }

// cos(2 pi j / 64) on [0, 16] (FP32, rounded from FP64; exact at 0 and 16)
__host__ __device__ constexpr float cos64q(int j) {
    return j == 0 ? 1.0f : j == 1 ? 0.9951847f : j == 2 ? 0.98078525f : j == 3 ? 0.95694035f
         : j == 4 ? 0.9238795f : j == 5 ? 0.8819213f : j == 6 ? 0.8314696f : j == 7 ? 0.77301043f
         : j == 8 ? 0.70710677f : j == 9 ? 0.6343933f : j == 10 ? 0.55557024f : j == 11 ? 0.47139674f
         : j == 12 ? 0.38268343f : j == 13 ? 0.29028466f : j == 14 ? 0.19509032f : j == 15 ? 0.09801714f
         : 0.0f;
}
__host__ __device__ constexpr float cos64(int j) {
    return (j & 63) <= 16 ? cos64q(j & 63)
         : (j & 63) <= 32 ? -cos64q(32 - (j & 63))
         : (j & 63) <= 48 ? -cos64q((j & 63) - 32)
         : cos64q(64 - (j & 63));
}
// W64^q = exp(-2 pi i q / 64)
__host__ __device__ constexpr float2 w64(int q) { return float2{cos64(q), -cos64((q + 48) & 63)}; }

// Cooperative async copy of rows [0, nrows) of columns col0, col0+1 of a
// [rows][nxh] array into the 2-column tile.
__device__ __forceinline__ void tile_load2(float2* tile, const float2* __restrict__ src, int nrows, int nxh,
                                           int col0) {
    for (int e = threadIdx.x; e < nrows * kW2Cols; e += 4 * 32) {
        const int i = e >> 1, c = e & 1;
        const bool ok = col0 + c < nxh;
        cp_async8(tile + tix2(i, c), src + (long long)i * nxh + (ok ? col0 + c : 0), ok);
    }
    cp_async_commit();
}

// X[1023 - f'] of the odd half from the lane holding it (f' = lane + 32 m):
// lane 31 - lane, register 31 - m.
__device__ __forceinline__ float2 warp_partner_rev(const float2 (&v)[32], int lane, int M) {
    float2 z;
    z.x = __shfl_sync(0xffffffffu, v[31 - M].x, 31 - lane);
    z.y = __shfl_sync(0xffffffffu, v[31 - M].y, 31 - lane);
    return z;
}

// The packed DC/Nyquist column: partner X[2048 - f] of f = 2 f' + par lies in
// the same half, at f'' = (1024 - f') mod 1024 (par 0) or 1023 - f' (par 1).
__device__ __forceinline__ void split2(const float2 (&v)[32], int lane, int M, int par, float2& A, float2& B) {
    const float2 zm = par ? warp_partner_rev(v, lane, M) : warp_partner(v, lane, M);
    split_dc_nyq(v[M], zm, A, B);
}

// F2 for Ny = 2048.  Grid (batch, ceil(NXh / 2)), 128 threads, kW2Smem bytes.
// hhT2: [m][NXh][2][1024] (par-split spectra of each column; c = 0 the DC
// column), hN2: [m][2][1024] (Nyquist column), tw2048l: W2048^l for l < 32.
template <typename HT = float2>
__global__ void __launch_bounds__(128, 3)
kw2_cols_fwd(const float2* __restrict__ Z, long long z_bstride, long long z_kstride,
             const HT* __restrict__ hhT2, const HT* __restrict__ hN2, const float* __restrict__ hscale, int m,
             const Box* __restrict__ box, int NXh, float2* __restrict__ A, long long a_bstride,
             const float2* __restrict__ tw, const float2* __restrict__ tw2048l, int* __restrict__ status,
             long long wait_limit, int skip_copy) {
    constexpr int NY = kW2N;
    extern __shared__ float2 smem[];
    float2* tile = smem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int par = warp & 1, cl = warp >> 1;
    float2* tr = smem + NY * kW2Cols + warp * kWarpN;
    const int b = blockIdx.x;
    const int col0 = blockIdx.y * kW2Cols;
    const int col = col0 + cl;
    const bool cv = col < NXh;
    const bool dcn = blockIdx.y == 0 && cl == 0;
    const float2* Zb = Z + b * z_bstride;
    __shared__ unsigned long long bars[4];
    unsigned long long* bar = &bars[warp];
    if (lane == 0) mbar_init(bar);
    __syncwarp();
    unsigned parity = 0;
    bool failed = false;
    const float2 wl = __ldg(&tw2048l[lane]);

    float2 acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = make_float2(0.f, 0.f);
    int k = 0;
    while (k < m && box[k].nr == 0) ++k;
    if (k < m) tile_load2(tile, Zb + k * z_kstride, box[k].nr, NXh, col0);
    while (k < m) {
        int kn = k + 1;
        while (kn < m && box[kn].nr == 0) ++kn;
        const Box bx = box[k];
        cp_async_wait_all();
        __syncthreads();
        float2 v[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int n = lane + 32 * q;
            const int i0 = wrap(n - bx.r0, NY), i1 = wrap(n + 1024 - bx.r0, NY);
            const float2 lo = (i0 < bx.nr) ? tile[tix2(i0, cl)] : make_float2(0.f, 0.f);
            const float2 hi = (i1 < bx.nr) ? tile[tix2(i1, cl)] : make_float2(0.f, 0.f);
            v[q] = par ? cmul(cmul(csub(lo, hi), wl), w64(q)) : cadd(lo, hi);
        }
        __syncthreads();
        if (kn < m) tile_load2(tile, Zb + kn * z_kstride, box[kn].nr, NXh, col0);
        const bool bulk = !dcn && cv && !failed;
        const float sk = hscale_of<HT>(hscale, k);
        warp_fft1024<false>(v, tr, tw, [&] {
            if (bulk && lane == 0)
                bulk_load(tr, hhT2 + (((long long)k * NXh + col) * 2 + par) * kWarpN, kWarpN * sizeof(HT), bar,
                          skip_copy);
        });
        if (bulk) {
            if (!mbar_wait(bar, parity, wait_limit)) {
                failed = true;
                if (lane == 0) atomicOr(status, kStatusTimeout);
                // a copy may still be in flight into the tile: wait for it once more
                mbar_wait(bar, parity, wait_limit);
            }
            parity ^= 1;
        }
        if (dcn) {
            const HT* h0 = hhT2 + (long long)k * NXh * 2 * kWarpN + par * kWarpN;
            const HT* hn = hN2 + ((long long)k * 2 + par) * kWarpN;
#pragma unroll
            for (int mm = 0; mm < 32; ++mm) {
                const int f = lane + 32 * mm;
                float2 a, bb;
                split2(v, lane, mm, par, a, bb);
                acc[mm] = cfma(ldh(&h0[f], sk), a, acc[mm]);
                const float2 t = cmul(ldh(&hn[f], sk), bb);
                acc[mm].x -= t.y;
                acc[mm].y += t.x;
            }
        } else if (cv && !failed) {
            const HT* th = reinterpret_cast<const HT*>(tr);
#pragma unroll
            for (int mm = 0; mm < 32; ++mm) acc[mm] = cfma(lds_h(&th[lane + 32 * mm], sk), v[mm], acc[mm]);
        }
        k = kn;
    }
    warp_fft1024<true>(acc, tr, tw);
    if (par) {
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = cmulc(cmulc(acc[q], wl), w64(q));
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 32; ++q) tile[tix2(lane + 32 * q + 1024 * par, cl)] = acc[q];
    __syncthreads();
    float2* Ab = A + b * a_bstride;
    for (int e = threadIdx.x; e < 1024 * kW2Cols; e += 4 * 32) {
        const int i = e >> 1, c = e & 1;
        if (col0 + c < NXh) {
            const float2 a = tile[tix2(i, c)], bq = tile[tix2(i + 1024, c)];
            Ab[(long long)i * NXh + col0 + c] = cadd(a, bq);
            Ab[(long long)(i + 1024) * NXh + col0 + c] = csub(a, bq);
        }
    }
}

// G2 for Ny = 2048 (box rows of each term's Q).  Grid (batch, ceil(NXh / 2)).
template <typename HT = float2>
__global__ void __launch_bounds__(128, 3)
kw2_cols_adj(const float2* __restrict__ V, long long v_bstride,
             const HT* __restrict__ hhT2, const HT* __restrict__ hN2, const float* __restrict__ hscale, int m,
             const Box* __restrict__ box, int NXh, float2* __restrict__ Q, long long q_bstride, long long q_kstride,
             const float2* __restrict__ tw, const float2* __restrict__ tw2048l, int* __restrict__ status,
             long long wait_limit, int skip_copy) {
    constexpr int NY = kW2N;
    extern __shared__ float2 smem[];
    float2* tile = smem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int par = warp & 1, cl = warp >> 1;
    float2* tr = smem + NY * kW2Cols + warp * kWarpN;
    const int b = blockIdx.x;
    const int col0 = blockIdx.y * kW2Cols;
    const int col = col0 + cl;
    const bool cv = col < NXh;
    const bool dcn = blockIdx.y == 0 && cl == 0;
    __shared__ unsigned long long bars[4];
    unsigned long long* bar = &bars[warp];
    if (lane == 0) mbar_init(bar);
    __syncwarp();
    unsigned parity = 0;
    bool failed = false;
    const bool use_bulk = !dcn && cv;
    const float2 wl = __ldg(&tw2048l[lane]);
    auto next_term = [&](int kk) {
        while (kk < m && box[kk].nr == 0) ++kk;
        return kk;
    };

    tile_load2(tile, V + b * v_bstride, NY, NXh, col0);
    cp_async_wait_all();
    __syncthreads();
    float2 vv[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const int n = lane + 32 * q;
        const float2 lo = tile[tix2(n, cl)], hi = tile[tix2(n + 1024, cl)];
        vv[q] = par ? cmul(cmul(csub(lo, hi), wl), w64(q)) : cadd(lo, hi);
    }
    int k = next_term(0);
    warp_fft1024<false>(vv, tr, tw, [&] {
        if (use_bulk && k < m && lane == 0)
            bulk_load(tr, hhT2 + (((long long)k * NXh + col) * 2 + par) * kWarpN, kWarpN * sizeof(HT), bar,
                      skip_copy);
    });
    while (k < m) {
        const Box bx = box[k];
        const int kn = next_term(k + 1);
        if (use_bulk && !failed) {
            if (!mbar_wait(bar, parity, wait_limit)) {
                failed = true;
                if (lane == 0) atomicOr(status, kStatusTimeout);
                mbar_wait(bar, parity, wait_limit);
            }
            parity ^= 1;
        }
        float2 p[32];
        const float sk = hscale_of<HT>(hscale, k);
        if (dcn) {
            const HT* h0 = hhT2 + (long long)k * NXh * 2 * kWarpN + par * kWarpN;
            const HT* hn = hN2 + ((long long)k * 2 + par) * kWarpN;
#pragma unroll
            for (int mm = 0; mm < 32; ++mm) {
                const int f = lane + 32 * mm;
                float2 a, bb;
                split2(vv, lane, mm, par, a, bb);
                float2 t = cmulc(a, ldh(&h0[f], sk));
                const float2 s = cmulc(bb, ldh(&hn[f], sk));
                t.x -= s.y;
                t.y += s.x;
                p[mm] = t;
            }
        } else {
            const HT* th = reinterpret_cast<const HT*>(tr);
#pragma unroll
            for (int mm = 0; mm < 32; ++mm)
                p[mm] = (use_bulk && !failed) ? cmulc(vv[mm], lds_h(&th[lane + 32 * mm], sk))
                                              : make_float2(0.f, 0.f);
        }
        const bool issue = use_bulk && !failed && kn < m;
        warp_fft1024<true, false>(p, tr, tw, [&] {
            if (issue && lane == 0)
                bulk_load(tr, hhT2 + (((long long)kn * NXh + col) * 2 + par) * kWarpN, kWarpN * sizeof(HT), bar,
                          skip_copy);
        });
        if (par) {
#pragma unroll
            for (int q = 0; q < 32; ++q) p[q] = cmulc(cmulc(p[q], wl), w64(q));
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 32; ++q) tile[tix2(lane + 32 * q + 1024 * par, cl)] = p[q];
        __syncthreads();
        float2* Qk = Q + b * q_bstride + k * q_kstride;
        for (int e = threadIdx.x; e < bx.nr * kW2Cols; e += 4 * 32) {
            const int i = e >> 1, c = e & 1;
            const int g = wrap(bx.r0 + i, NY);
            if (col0 + c < NXh) {
                const int g0 = g & 1023;
                const float2 a = tile[tix2(g0, c)], bq = tile[tix2(g0 + 1024, c)];
                Qk[(long long)i * NXh + col0 + c] = g < 1024 ? cadd(a, bq) : csub(a, bq);
            }
        }
        k = kn;
    }
}

}  // namespace pce
