// warpfft.cuh -- one-warp 1024-point FFT (four-step, 32 x 32) for sm_103a.
//
// Lane l holds v[q] = x[l + 32 q] (q = 0..31).  With n = l + 32 q and
// k = p + 32 m (l, q, p, m < 32):
//   X[p + 32 m] = sum_l W32^{l m} W1024^{l p} sum_q x[l + 32 q] W32^{q p},
// so the FFT is
//   1. a 32-point DFT over q in each lane's registers,
//   2. the twiddles W1024^{l p} (table, FP32 rounded from FP64),
//   3. a transpose of the 32 x 32 block through a warp-private shared tile
//      (XOR-swizzled: element (l, p) at l*32 + (p ^ l), conflict-free both
//      for the column writes and the row reads of a half-warp),
//   4. a 32-point DFT over l in each lane.
// On exit lane p holds v[m] = X[p + 32 m]: the same layout as on entry, so a
// forward FFT, a pointwise product and an inverse FFT chain in registers.
// Only __syncwarp is used: warps never wait for one another.
// The inverse uses the conjugate twiddles and is unnormalised.
#pragma once

#include "fft.cuh"

namespace pce {

// cos(2 pi j / 32) on [0, 8] (FP32, correctly rounded; exact at 0 and 8)
__host__ __device__ constexpr float cos32q(int j) {
    return j == 0 ? 1.0f
         : j == 1 ? 0.980785251f
         : j == 2 ? 0.923879504f
         : j == 3 ? 0.831469595f
         : j == 4 ? 0.707106769f
         : j == 5 ? 0.555570245f
         : j == 6 ? 0.382683426f
         : j == 7 ? 0.195090324f
         : 0.0f;
}
__host__ __device__ constexpr float cos32(int j) {
    return (j & 31) <= 8 ? cos32q(j & 31)
         : (j & 31) <= 16 ? -cos32q(16 - (j & 31))
         : (j & 31) <= 24 ? -cos32q((j & 31) - 16)
         : cos32q(32 - (j & 31));
}
// sin(2 pi j / 32) = cos(2 pi (j - 8) / 32)
__host__ __device__ constexpr float sin32(int j) { return cos32((j + 24) & 31); }

// x * W32^j (forward: exp(-2 pi i j / 32); inverse: conjugate); j a compile-time constant
template <bool INV>
__device__ __forceinline__ float2 tw32(float2 x, int j) {
    if (j == 0) return x;
    if (j == 8) return mul_mi<INV>(x);
    const float c = cos32(j);
    const float s = INV ? sin32(j) : -sin32(j);
    return cmul(x, make_float2(c, s));
}

// 8-point DFT of x[0..3] with x[4..7] = 0 (the first decimation-in-frequency
// butterflies of Dft<8> reduce to copies).
template <bool INV>
__device__ __forceinline__ void dft8_lower_half(float2 (&a)[8]) {
    const float h = 0.70710678118654752440f;
    float2 b[4], e[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = e[q] = a[q];
    {
        float2 x = e[1];
        e[1] = INV ? make_float2((x.x - x.y) * h, (x.x + x.y) * h) : make_float2((x.x + x.y) * h, (x.y - x.x) * h);
        e[2] = mul_mi<INV>(e[2]);
        x = e[3];
        e[3] = INV ? make_float2((-x.x - x.y) * h, (x.x - x.y) * h) : make_float2((x.y - x.x) * h, (-x.x - x.y) * h);
    }
    Dft<4, INV>::run(b);
    Dft<4, INV>::run(e);
    a[0] = b[0]; a[2] = b[1]; a[4] = b[2]; a[6] = b[3];
    a[1] = e[0]; a[3] = e[1]; a[5] = e[2]; a[7] = e[3];
}

// Outputs 0 and 1 of the 4-point DFT only.
template <bool INV>
__device__ __forceinline__ void dft4_first_two(float2 (&a)[4]) {
    const float2 d0 = cadd(a[0], a[2]);
    const float2 d1 = csub(a[0], a[2]);
    const float2 d2 = cadd(a[1], a[3]);
    const float2 d3 = mul_mi<INV>(csub(a[1], a[3]));
    a[0] = cadd(d0, d2);
    a[1] = cadd(d1, d3);
}

// In-register 32-point DFT, natural order in and out: n = 4 n1 + n2,
// k = k1 + 8 k2, X[k1 + 8 k2] = sum_n2 W4^{n2 k2} W32^{n2 k1} sum_n1 x[4 n1 + n2] W8^{n1 k1}.
// IN_HALF: x[16..31] are zero (n1 >= 4) and are not read.
// OUT_HALF: only X[0..15] (k2 < 2) are computed; a[16..31] are left undefined.
template <bool INV, bool IN_HALF = false, bool OUT_HALF = false>
__device__ __forceinline__ void dft32(float2 (&a)[32]) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        float2 x[8];
        if constexpr (IN_HALF) {
#pragma unroll
            for (int n1 = 0; n1 < 4; ++n1) x[n1] = a[4 * n1 + n2];
            dft8_lower_half<INV>(x);
        } else {
#pragma unroll
            for (int n1 = 0; n1 < 8; ++n1) x[n1] = a[4 * n1 + n2];
            Dft<8, INV>::run(x);
        }
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) a[4 * k1 + n2] = tw32<INV>(x[k1], n2 * k1);
    }
    float2 out[32];
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
        float2 y[4] = {a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]};
        if constexpr (OUT_HALF) {
            dft4_first_two<INV>(y);
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2) out[k1 + 8 * k2] = y[k2];
        } else {
            Dft<4, INV>::run(y);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) out[k1 + 8 * k2] = y[k2];
        }
    }
#pragma unroll
    for (int i = 0; i < (OUT_HALF ? 16 : 32); ++i) a[i] = out[i];
}

// Twiddle table of the four-step 1024-point FFT: tw[p * 32 + l] = W1024^{l p}.
constexpr int kWarpTwLen = 1024;

struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// One-warp 1024-point FFT (see the file comment).  tile: 1024 float2 of
// shared memory private to the calling warp.  All 32 lanes must call it.
// hook() runs once the transpose has been read back, i.e. when the tile is
// free again (it may start an asynchronous copy into the tile).
// SPLIT: the twiddles W1024^{l p} come from ten table loads and products (fewer
// loads in flight, more multiplies); otherwise from 31 table loads.  Which one
// is faster depends on the register pressure of the calling kernel.
// IN_HALF: the inputs x[l + 32 q] with q >= 16 are zero (v[16..31] not read).
// OUT_HALF: only the outputs X[p + 32 m] with m < 16 are computed (v[16..31]
// undefined on exit).
template <bool INV, bool SPLIT = true, typename Hook = NoHook, bool IN_HALF = false, bool OUT_HALF = false>
__device__ __forceinline__ void warp_fft1024(float2 (&v)[32], float2* tile, const float2* __restrict__ tw,
                                             Hook hook = Hook()) {
    const int lane = threadIdx.x & 31;
    dft32<INV, IN_HALF>(v);
    // keep the twiddle loads after the first DFT: hoisted above it they would
    // hold 62 more registers through it
    __syncwarp();
    if constexpr (SPLIT) {
        // W1024^{l p} with p = 8 a + b is W1024^{8 l a} W1024^{l b}: ten table
        // loads issued together, then products (two roundings at most)
        float2 wb[8], wa[4];
#pragma unroll
        for (int q = 1; q < 8; ++q) wb[q] = __ldg(&tw[q * 32 + lane]);
#pragma unroll
        for (int q = 1; q < 4; ++q) wa[q] = __ldg(&tw[8 * q * 32 + lane]);
#pragma unroll
        for (int p = 1; p < 32; ++p) {
            const int a = p >> 3, bq = p & 7;
            const float2 t = a == 0 ? wb[bq] : (bq == 0 ? wa[a] : cmul(wa[a], wb[bq]));
            v[p] = INV ? cmulc(v[p], t) : cmul(v[p], t);
        }
    } else {
#pragma unroll
        for (int p = 1; p < 32; ++p) {
            const float2 t = __ldg(&tw[p * 32 + lane]);
            v[p] = INV ? cmulc(v[p], t) : cmul(v[p], t);
        }
    }
    __syncwarp();
#pragma unroll
    for (int p = 0; p < 32; ++p) tile[lane * 32 + (p ^ lane)] = v[p];
    __syncwarp();
#pragma unroll
    for (int l = 0; l < 32; ++l) v[l] = tile[l * 32 + (lane ^ l)];
    __syncwarp();
    hook();
    dft32<INV, false, OUT_HALF>(v);
}

// In-register 16-point DFT, natural order in and out: n = 4 n1 + n2,
// k = k1 + 4 k2, X[k1 + 4 k2] = sum_n2 W4^{n2 k2} W16^{n2 k1} sum_n1 x[4 n1 + n2] W4^{n1 k1}.
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&a)[16]) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        float2 x[4] = {a[n2], a[4 + n2], a[8 + n2], a[12 + n2]};
        Dft<4, INV>::run(x);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) a[4 * k1 + n2] = tw32<INV>(x[k1], 2 * n2 * k1);   // W16 = W32^2
    }
    float2 out[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 y[4] = {a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]};
        Dft<4, INV>::run(y);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) out[k1 + 4 * k2] = y[k2];
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = out[i];
}

// One-warp 512-point FFT with the layout of warp_fft1024: lane l holds
// v[q] = x[l + 32 q] (q < 16) on entry and v[m] = X[l + 32 m] on exit.  With
// n = l + 32 q and k = p + 16 j (p < 16, j < 32):
//   X[p + 16 j] = sum_l W32^{l j} W512^{l p} sum_q x[l + 32 q] W16^{q p},
//   1. a 16-point DFT over q in each lane's registers,
//   2. the twiddles W512^{l p} = W1024^{2 l p} (the 1024-point table, rows 2p),
//   3. the 32 x 16 block y[l][p] through a warp-private shared tile (the 16
//      entries of row l XOR-swizzled by l & 15: conflict-free per half-warp),
//   4. the 32-point DFTs over l, one per p, split by decimation in frequency
//      over the lane pair (p, p + 16): lane p + 16 s forms
//      a_s[l'] = (y[l'][p] + (-1)^s y[l' + 16][p]) W32^{s l'} (l' < 16) from the
//      tile and takes its 16-point DFT, which gives X[p + 16 (2 j' + s)]
//      = X[lane + 32 j'] (j' < 16): the natural layout again.
// tile: 512 float2 private to the warp.  Hook and SPLIT as for warp_fft1024.
template <bool INV, bool SPLIT = true, typename Hook = NoHook>
__device__ __forceinline__ void warp_fft512(float2 (&v)[16], float2* tile, const float2* __restrict__ tw,
                                            Hook hook = Hook()) {
    const int lane = threadIdx.x & 31;
    dft16<INV>(v);
    __syncwarp();
    if constexpr (SPLIT) {
        // W512^{l p}, p = 8 a + b: W1024^{16 l a} W1024^{2 l b}
        float2 wb[8], wa;
#pragma unroll
        for (int q = 1; q < 8; ++q) wb[q] = __ldg(&tw[2 * q * 32 + lane]);
        wa = __ldg(&tw[16 * 32 + lane]);
#pragma unroll
        for (int p = 1; p < 16; ++p) {
            const int bq = p & 7;
            const float2 t = p < 8 ? wb[bq] : (bq == 0 ? wa : cmul(wa, wb[bq]));
            v[p] = INV ? cmulc(v[p], t) : cmul(v[p], t);
        }
    } else {
#pragma unroll
        for (int p = 1; p < 16; ++p) {
            const float2 t = __ldg(&tw[2 * p * 32 + lane]);
            v[p] = INV ? cmulc(v[p], t) : cmul(v[p], t);
        }
    }
    __syncwarp();
#pragma unroll
    for (int p = 0; p < 16; ++p) tile[lane * 16 + (p ^ (lane & 15))] = v[p];
    __syncwarp();
    const int p = lane & 15;
    const bool odd = lane >= 16;
    const float sg = odd ? -1.f : 1.f;
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        const float2 y0 = tile[l * 16 + (p ^ l)];
        const float2 y1 = tile[(l + 16) * 16 + (p ^ l)];
        float2 a = make_float2(fmaf(sg, y1.x, y0.x), fmaf(sg, y1.y, y0.y));
        if (l > 0 && odd) a = tw32<INV>(a, l);
        v[l] = a;
    }
    __syncwarp();
    hook();
    dft16<INV>(v);
}

// One-warp FFT of NY = 512 or 1024 points (NY / 32 values per lane).
template <int NY, bool INV, bool SPLIT = true, typename Hook = NoHook>
__device__ __forceinline__ void warp_fft(float2 (&v)[NY / 32], float2* tile, const float2* __restrict__ tw,
                                         Hook hook = Hook()) {
    static_assert(NY == 512 || NY == 1024, "one-warp FFT of 512 or 1024 points");
    if constexpr (NY == 1024) warp_fft1024<INV, SPLIT, Hook>(v, tile, tw, hook);
    else warp_fft512<INV, SPLIT, Hook>(v, tile, tw, hook);
}

// Value X[NY - f] for f = lane + 32 m (NY = 32 Q), from the lane holding it:
// lane (32 - lane) & 31, register Q - 1 - m; lane 0 holds its own partner in
// register (Q - m) & (Q - 1).
template <int Q>
__device__ __forceinline__ float2 warp_partner(const float2 (&v)[Q], int lane, int M) {
    float2 z;
    z.x = __shfl_sync(0xffffffffu, v[Q - 1 - M].x, (32 - lane) & 31);
    z.y = __shfl_sync(0xffffffffu, v[Q - 1 - M].y, (32 - lane) & 31);
    if (lane == 0) z = v[(Q - M) & (Q - 1)];
    return z;
}

}  // namespace pce
