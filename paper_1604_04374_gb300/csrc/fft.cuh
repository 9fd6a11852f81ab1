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
// shared-memory buffer: one float2 of padding per 16, so that every write
// and read pattern of the stages touches each 8-byte bank pair exactly twice
// per warp (two wavefronts, the minimum for 64-bit accesses), also when one
// warp spans several FFTs whose buffers are staggered by 4 float2.
//
// Twiddles come from a per-N table generated once per plan in FP64 and
// rounded to FP32 (layout: per stage s >= 1, entries [q-1][k] =
// exp(-2 i pi q k / (Ns Rs)), k fastest).  The forward transform uses the
// sign of the Fourier atoms exp(-2 i pi k x) (Section 2); the inverse uses
// the conjugate twiddles and is unnormalised.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pce {

constexpr int kR = 8;   // elements per thread

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int pad_len(int n) { return n + (n >> 4); }
// Shared-memory float2 count of one FFT's two buffers plus the skew that
// staggers neighbouring FFTs by 32 bytes (8 banks).
__host__ __device__ constexpr int fft_region(int n) { return 2 * pad_len(n) + 4; }

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

// One Stockham stage.  buf: one of this FFT's two shared buffers (pad_len(N) float2).
template <int N, int S, bool INV>
__device__ __forceinline__ void fft_stage(float2 (&v)[kR], int j, float2* buf,
                                          const float2* __restrict__ tw) {
    using P = FftPlan<N>;
    constexpr int RS = P::radix(S);
    constexpr int NS = P::ns(S);
    constexpr int G = kR / RS;
    constexpr bool LAST = (S == P::NSTAGES - 1);
    constexpr int T = P::T;
#pragma unroll
    for (int i = 0; i < G; ++i) {
        const int jp = j + i * T;
        const int k = jp & (NS - 1);
        float2 a[RS];
#pragma unroll
        for (int q = 0; q < RS; ++q) a[q] = v[i + q * G];
        if (S > 0) {
#pragma unroll
            for (int q = 1; q < RS; ++q) {
                const float2 t = __ldg(&tw[P::twoff(S) + (q - 1) * NS + k]);
                a[q] = INV ? cmulc(a[q], t) : cmul(a[q], t);
            }
        }
        Dft<RS, INV>::run(a);
        if (LAST) {
#pragma unroll
            for (int q = 0; q < RS; ++q) v[i + q * G] = a[q];
        } else {
            // padded address of base + q NS, strength-reduced: the low four bits
            // of base + q NS only come from k (NS >= 16), from k < 8 plus 8 q
            // (NS = 8), or from q < 8 on base = 8 jp (NS = 1)
            const int base = (jp / NS) * NS * RS + k;
            const int pb = padi(base);
#pragma unroll
            for (int q = 0; q < RS; ++q) {
                int addr;
                if constexpr (NS >= 16) addr = pb + q * (NS + NS / 16);
                else if constexpr (NS == 8) addr = pb + 8 * q + (q >> 1);
                else if constexpr (NS == 1 && RS == kR) addr = pb + q;
                else addr = padi(base + q * NS);
                buf[addr] = a[q];
            }
        }
    }
    if (!LAST) {
        __syncthreads();
        if constexpr (T % 16 == 0) {
            const int pj = padi(j);
#pragma unroll
            for (int r = 0; r < kR; ++r) v[r] = buf[pj + r * (T + T / 16)];
        } else {
#pragma unroll
            for (int r = 0; r < kR; ++r) v[r] = buf[padi(j + r * T)];
        }
    }
}

template <int N, int S, bool INV>
struct FftStages {
    __device__ __forceinline__ static void run(float2 (&v)[kR], int j, float2* b0, float2* b1,
                                               const float2* __restrict__ tw) {
        fft_stage<N, S, INV>(v, j, (S & 1) ? b1 : b0, tw);
        FftStages<N, S + 1, INV>::run(v, j, b0, b1, tw);
    }
};
template <int N, bool INV>
struct FftStages<N, FftPlan<N>::NSTAGES, INV> {
    __device__ __forceinline__ static void run(float2 (&)[kR], int, float2*, float2*,
                                               const float2* __restrict__) {}
};

// Complex FFT of N points held as v[r] = x[j + r*T] by threads j = 0..T-1.
// b0, b1: two shared buffers of pad_len(N) float2 private to this FFT.
// Begins with a CTA barrier so that the buffers may be reused freely by the
// caller between FFTs.  All threads of the CTA must call it.
template <int N, bool INV>
__device__ __forceinline__ void fft(float2 (&v)[kR], int j, float2* b0, float2* b1,
                                    const float2* __restrict__ tw) {
    __syncthreads();
    FftStages<N, 0, INV>::run(v, j, b0, b1, tw);
}

}  // namespace pce
