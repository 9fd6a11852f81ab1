// fft.cuh -- shared-memory Stockham FFT core for sm_103a.
//
// One complex FFT of length N (power of two) is executed by T = N/R threads
// of a CTA, each holding R = 8 elements in registers.  Thread j holds the
// elements j + r*T (r = 0..R-1) on entry AND on exit (natural order), so
// an FFT, a pointwise multiply and an inverse FFT chain from registers.
//
// Stages are Stockham autosort radix-8 stages with one smaller radix (2 or 4)
// last when log2(N) is not a multiple of 3.  Stage s with radix Rs and
// current sub-transform length Ns: butterfly j' reads x[j' + q N/Rs], applies
// the twiddles W_{Ns Rs}^{q k} (k = j' mod Ns) and writes
// y[(j'/Ns) Ns Rs + k + q Ns].  Between stages data goes through a padded
// shared-memory buffer, alternating between two buffers.  64-bit shared
// accesses are serviced per half-warp, so a half-warp's 16 lanes must hit 16
// distinct 8-byte bank pairs; the padding is chosen per exchange for the two
// thread layouts the kernels use:
//   kRowLayout: a half-warp is 16 consecutive j of one FFT.  The exchange
//     after stage 0 (writes with stride 8) and after stages >= 2 (contiguous
//     writes) pads one float2 per 16; the exchange after stage 1 (two runs
//     of 8 that lie 64 apart) shifts every 64-element block by 8.
//   kColLayout: a half-warp is 4 consecutive j of 4 FFTs whose buffers are
//     staggered by 4 float2: one float2 of padding per 8 throughout.
// The twiddles of a stage are loaded before the barrier that precedes it, so
// their latency overlaps the exchange.
//
// Twiddles come from a per-N table generated once per plan in FP64 and
// rounded to FP32 (layout: per stage s >= 1, entries [q-1][k] =
// exp(-2 i pi q k / (Ns Rs)), k fastest).  The forward transform uses the
// sign of the Fourier atoms exp(-2 i pi k x) (Section 2); the inverse uses
// the conjugate twiddles and is unnormalised.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pce {

// ---- storage precision of windows (W) and spectra (H)
// FP32 storage: float windows, float2 spectra.  Reduced storage: bfloat16
// windows, half2 spectra scaled per term by a power of two.  Loads convert
// to FP32; all arithmetic is FP32.
__device__ __forceinline__ float ldw(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldw(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float2 ldh(const float2* p, float) { return __ldg(p); }
__device__ __forceinline__ float2 ldh(const __half2* p, float s) {
    const float2 f = __half22float2(__ldg(p));
    return make_float2(f.x * s, f.y * s);
}
// the same from shared memory
__device__ __forceinline__ float2 lds_h(const float2* p, float) { return *p; }
__device__ __forceinline__ float2 lds_h(const __half2* p, float s) {
    const float2 f = __half22float2(*p);
    return make_float2(f.x * s, f.y * s);
}
template <typename HT>
__device__ __forceinline__ float hscale_of(const float* hscale, int k) {
    return sizeof(HT) == sizeof(float2) ? 1.f : __ldg(&hscale[k]);
}

constexpr int kR = 8;   // elements per thread

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

enum FftLayout { kRowLayout = 0, kColLayout = 1 };

// Generic padding used outside the stages (one float2 per 16).
__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }
// float2 count of one exchange buffer (room for every exchange's padding).
__host__ __device__ constexpr int pad_len(int n) { return n + n / 8 + 8; }
// One FFT's two buffers plus a 4-float2 skew that staggers neighbouring FFTs.
__host__ __device__ constexpr int fft_region(int n) { return 2 * pad_len(n) + 4; }

// Address of element i in the buffer written by stage E.
template <int L, int E>
__device__ __forceinline__ int xaddr(int i) {
    if constexpr (L == kColLayout) return i + (i >> 3);
    else if constexpr (E == 1) return i + ((i >> 6) << 3);
    else return i + (i >> 4);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// acc + a * b
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
// acc + conj(a) * b
__device__ __forceinline__ float2 cfmac(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// In-register DFT of RS points, natural order in and out.
template <int RS, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
    __device__ __forceinline__ static void run(float2* a) {
        float2 t = csub(a[0], a[1]);
        a[0] = cadd(a[0], a[1]);
        a[1] = t;
    }
};

template <bool INV>
struct Dft<4, INV> {
    __device__ __forceinline__ static void run(float2* a) {
        float2 d0 = cadd(a[0], a[2]);
        float2 d1 = csub(a[0], a[2]);
        float2 d2 = cadd(a[1], a[3]);
        float2 d3 = mul_mi<INV>(csub(a[1], a[3]));
        a[0] = cadd(d0, d2);
        a[2] = csub(d0, d2);
        a[1] = cadd(d1, d3);
        a[3] = csub(d1, d3);
    }
};

template <bool INV>
struct Dft<8, INV> {
    __device__ __forceinline__ static void run(float2* a) {
        const float h = 0.70710678118654752440f;
        float2 b[4], e[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            b[q] = cadd(a[q], a[q + 4]);
            e[q] = csub(a[q], a[q + 4]);
        }
        // e[q] *= W8^q
        {
            float2 x = e[1];
            e[1] = INV ? make_float2((x.x - x.y) * h, (x.x + x.y) * h)
                       : make_float2((x.x + x.y) * h, (x.y - x.x) * h);
            e[2] = mul_mi<INV>(e[2]);
            x = e[3];
            e[3] = INV ? make_float2((-x.x - x.y) * h, (x.x - x.y) * h)
                       : make_float2((x.y - x.x) * h, (-x.x - x.y) * h);
        }
        Dft<4, INV>::run(b);
        Dft<4, INV>::run(e);
        a[0] = b[0]; a[2] = b[1]; a[4] = b[2]; a[6] = b[3];
        a[1] = e[0]; a[3] = e[1]; a[5] = e[2]; a[7] = e[3];
    }
};

// Compile-time description of the stage sequence for an N-point FFT.
template <int N>
struct FftPlan {
    static constexpr int R = kR;
    static constexpr int T = N / R;
    static constexpr int L = ilog2(N);
    static constexpr int LR = ilog2(R);
    static constexpr int NFULL = L / LR;
    static constexpr int REM = L % LR;
    static constexpr int NSTAGES = NFULL + (REM ? 1 : 0);
    __host__ __device__ static constexpr int radix(int s) { return s < NFULL ? R : (1 << REM); }
    __host__ __device__ static constexpr int ns(int s) { return 1 << (LR * s); }
    // offset of stage s's twiddles in the table (stages 1..NSTAGES-1)
    __host__ __device__ static constexpr int twoff(int s) {
        return s <= 1 ? 0 : twoff(s - 1) + (radix(s - 1) - 1) * ns(s - 1);
    }
    static constexpr int TWLEN = twoff(NSTAGES);
    static_assert(N >= 16, "FFT length must be at least 16");
    static_assert((N & (N - 1)) == 0, "FFT length must be a power of two");
};

// Twiddles one thread applies in stage S (S >= 1): G butterflies x (RS - 1).
template <int N, int S>
__device__ __forceinline__ void load_tw(float2 (&t)[kR - 1], int j, const float2* __restrict__ tw) {
    using P = FftPlan<N>;
    constexpr int RS = P::radix(S);
    constexpr int NS = P::ns(S);
    constexpr int G = kR / RS;
#pragma unroll
    for (int i = 0; i < G; ++i) {
        const int k = (j + i * P::T) & (NS - 1);
#pragma unroll
        for (int q = 1; q < RS; ++q) t[i * (RS - 1) + q - 1] = __ldg(&tw[P::twoff(S) + (q - 1) * NS + k]);
    }
}

// Stage S of the FFT and, by recursion, every later stage.  t holds this
// stage's twiddles (unused for S = 0).
template <int N, int S, bool INV, int L>
__device__ __forceinline__ void fft_stage(float2 (&v)[kR], int j, float2* b0, float2* b1,
                                          const float2 (&t)[kR - 1], const float2* __restrict__ tw) {
    using P = FftPlan<N>;
    constexpr int RS = P::radix(S);
    constexpr int NS = P::ns(S);
    constexpr int G = kR / RS;
    constexpr bool LAST = (S == P::NSTAGES - 1);
    constexpr int T = P::T;
    float2* buf = (S & 1) ? b1 : b0;
#pragma unroll
    for (int i = 0; i < G; ++i) {
        const int jp = j + i * T;
        const int k = jp & (NS - 1);
        float2 a[RS];
#pragma unroll
        for (int q = 0; q < RS; ++q) a[q] = v[i + q * G];
        if constexpr (S > 0) {
#pragma unroll
            for (int q = 1; q < RS; ++q)
                a[q] = INV ? cmulc(a[q], t[i * (RS - 1) + q - 1]) : cmul(a[q], t[i * (RS - 1) + q - 1]);
        }
        Dft<RS, INV>::run(a);
        if constexpr (LAST) {
#pragma unroll
            for (int q = 0; q < RS; ++q) v[i + q * G] = a[q];
        } else {
            // address of base + q NS, strength-reduced where the padding allows
            const int base = (jp / NS) * NS * RS + k;
            const int pb = xaddr<L, S>(base);
#pragma unroll
            for (int q = 0; q < RS; ++q) {
                int addr;
                if constexpr (L == kColLayout && NS >= 8) addr = pb + q * (NS + NS / 8);
                else if constexpr (L == kRowLayout && S != 1 && NS >= 16) addr = pb + q * (NS + NS / 16);
                else if constexpr (L == kRowLayout && S == 1 && NS == 8 && RS == kR) addr = pb + 8 * q;
                else if constexpr (NS == 1 && RS == kR) addr = pb + q;
                else addr = xaddr<L, S>(base + q * NS);
                buf[addr] = a[q];
            }
        }
    }
    if constexpr (!LAST) {
        float2 tn[kR - 1];
        load_tw<N, S + 1>(tn, j, tw);
        __syncthreads();
        if constexpr (L == kColLayout && T % 8 == 0) {
            const int pj = xaddr<L, S>(j);
#pragma unroll
            for (int r = 0; r < kR; ++r) v[r] = buf[pj + r * (T + T / 8)];
        } else if constexpr (L == kRowLayout && S == 1 && T % 64 == 0) {
            const int pj = xaddr<L, S>(j);
#pragma unroll
            for (int r = 0; r < kR; ++r) v[r] = buf[pj + r * (T + T / 8)];
        } else if constexpr (L == kRowLayout && S != 1 && T % 16 == 0) {
            const int pj = xaddr<L, S>(j);
#pragma unroll
            for (int r = 0; r < kR; ++r) v[r] = buf[pj + r * (T + T / 16)];
        } else {
#pragma unroll
            for (int r = 0; r < kR; ++r) v[r] = buf[xaddr<L, S>(j + r * T)];
        }
        fft_stage<N, S + 1, INV, L>(v, j, b0, b1, tn, tw);
    }
}

// Complex FFT of N points held as v[r] = x[j + r*T] by threads j = 0..T-1.
// b0, b1: two shared buffers of pad_len(N) float2 private to this FFT.
// Begins with a CTA barrier so that the buffers may be reused freely by the
// caller between FFTs.  All threads of the CTA must call it.
template <int N, bool INV, int L = kRowLayout>
__device__ __forceinline__ void fft(float2 (&v)[kR], int j, float2* b0, float2* b1,
                                    const float2* __restrict__ tw) {
    float2 t0[kR - 1];
    __syncthreads();
    fft_stage<N, 0, INV, L>(v, j, b0, b1, t0, tw);
}

}  // namespace pce
