// k1d_large.cuh -- 1D transforms longer than one CTA holds (N = NY * NX,
// N > 8192), as a four-step FFT over the NY x NX view of a sequence
// (n = c + NX r: row r, column c):
//   X[a + NY b] = sum_c W_NX^{c b} [ W_N^{c a} sum_r x[c + NX r] W_NY^{r a} ],
// i.e. column FFTs, the twiddles W_N^{c a}, row FFTs.  The spectrum stays in
// this order (element a + NY b at row a, column b): the products with the
// spectra of h_k are pointwise, so no transpose is ever needed, and the
// inverse runs the same steps backwards (row IFFTs, conjugate twiddles,
// column IFFTs).  h_k's spectra are kept in the same order, in full (N
// complex values per term).
//
// Forward apply (per right-hand side b; two terms per complex FFT):
//   K1 k4_cols<MODE_WIN>:  G_p = twiddled column FFTs of w_{2p} u + i w_{2p+1} u
//   K2 k4_rows_fwd:        per row pair (a, NY - a): row FFTs of G_p, separation of
//                          the two terms' spectra, times hhat, accumulated over p
//                          on chip; then row IFFTs and conjugate twiddles
//   K3 k4_cols_inv:        column IFFTs, real part, / N
// Adjoint: K1<MODE_ONE> on v, K2' k4_rows_adj (row FFT once, per pair the
// products with conj(hhat) and row IFFTs), K3' k4_cols_adj (per pair column
// IFFTs, times w, accumulated).
#pragma once

#include "kernels.cuh"

namespace pce {

enum { kL1Win = 0, kL1Pair = 1, kL1One = 2 };

// K1.  Grid (npairs or 1, batch, NX / C).  Output G[(b * npairs + p)][a][c]
// = W_N^{c a} * FFT_r(x[c + NX r])[a], with x per MODE:
//   kL1Win : w_{2p} . src_b + i w_{2p+1} . src_b  (w dense [m][N], m terms)
//   kL1Pair: src[2p] + i src[2p + 1]               (src [m][N])
//   kL1One : src_b + 0 i
template <int NY, int MODE>
__global__ void __launch_bounds__(ColCfg<NY>::NT)
k4_cols(const float* __restrict__ src, long long src_bstride, const float* __restrict__ w, int m, int NX,
        const float2* __restrict__ twN, float2* __restrict__ G, const float2* __restrict__ tw) {
    using CC = ColCfg<NY>;
    constexpr int T = CC::T;
    constexpr int C = CC::C;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % C;
    const int j = threadIdx.x / C;
    float2* b0 = smem + c * CC::CS;
    float2* b1 = b0 + pad_len(NY);
    const int p = blockIdx.x;
    const int b = blockIdx.y;
    const int npairs = gridDim.x;
    const int col = blockIdx.z * C + c;
    const bool cv = col < NX;
    const long long N = (long long)NY * NX;
    const int k0 = 2 * p, k1 = 2 * p + 1;
    const bool has1 = MODE == kL1One ? false : (k1 < m);
    float2 v[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const long long n = col + (long long)NX * (j + r * T);
        float re = 0.f, im = 0.f;
        if (cv) {
            if (MODE == kL1Win) {
                const float s = __ldg(src + b * src_bstride + n);
                re = __ldg(w + (long long)k0 * N + n) * s;
                im = has1 ? __ldg(w + (long long)k1 * N + n) * s : 0.f;
            } else if (MODE == kL1Pair) {
                re = __ldg(src + (long long)k0 * N + n);
                im = has1 ? __ldg(src + (long long)k1 * N + n) : 0.f;
            } else {
                re = __ldg(src + b * src_bstride + n);
            }
        }
        v[r] = make_float2(re, im);
    }
    fft<NY, false, kColLayout>(v, j, b0, b1, tw);
    if (cv) {
        float2* Gu = G + ((long long)b * npairs + p) * N;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int a = j + r * T;
            Gu[(long long)a * NX + col] = cmul(v[r], __ldg(&twN[(long long)col * a]));
        }
    }
}

// Row-pair kernels: an item is the pair of rows (a, (NY - a) mod NY),
// a = 0 .. NY/2; each row is one FFT group of T = NX/8 threads.
template <int NX>
struct L1Rows {
    static constexpr int T = NX / kR;
    static constexpr int ITEMS = (256 / (2 * T)) > 0 ? 256 / (2 * T) : 1;   // row pairs per CTA
    static constexpr int NT = 2 * T * ITEMS;
    static constexpr int SMEM = 2 * ITEMS * fft_region(NX) * (int)sizeof(float2);
};

// Partner column of (a, col) in the spectrum order: X[N - f] for f = a + NY col
// sits at (NY - a, NX - 1 - col) when a != 0, at (0, (NX - col) mod NX) when a = 0.
__device__ __forceinline__ int l1_partner_col(int a, int col, int NX) {
    return a != 0 ? NX - 1 - col : (NX - col) & (NX - 1);
}

// K2.  Grid (ceil((NY/2 + 1) / ITEMS), batch).  Writes A[b][a][c] = conjugate
// twiddle times the row IFFT of sum_k hhat_k . X_k (rows a and NY - a).
template <int NX>
__global__ void __launch_bounds__(L1Rows<NX>::NT)
k4_rows_fwd(const float2* __restrict__ G, int npairs, const float2* __restrict__ hh4, int m, int NY,
            const float2* __restrict__ twN, float2* __restrict__ A, const float2* __restrict__ tw) {
    using L = L1Rows<NX>;
    constexpr int T = L::T;
    extern __shared__ float2 smem[];
    const int grp = threadIdx.x / T;           // 0 .. 2*ITEMS-1
    const int j = threadIdx.x - grp * T;
    const int item = grp >> 1, side = grp & 1;
    float2* b0 = smem + grp * fft_region(NX);
    float2* b1 = b0 + pad_len(NX);
    float2* pb0 = smem + (grp ^ 1) * fft_region(NX);   // partner row's buffer
    const int a0 = blockIdx.x * L::ITEMS + item;
    const bool active = a0 <= NY / 2;
    const int a = side == 0 ? (active ? a0 : 0) : ((NY - (active ? a0 : 0)) & (NY - 1));
    const int b = blockIdx.y;
    const long long N = (long long)NY * NX;
    float2 acc[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) acc[r] = make_float2(0.f, 0.f);
    for (int p = 0; p < npairs; ++p) {
        const float2* Gr = G + ((long long)b * npairs + p) * N + (long long)a * NX;
        float2 v[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) v[r] = __ldg(&Gr[j + r * T]);
        fft<NX, false>(v, j, b0, b1, tw);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kR; ++r) b0[padi(j + r * T)] = v[r];
        __syncthreads();
        const int k0 = 2 * p, k1 = 2 * p + 1;
        const float2* h0 = hh4 + (long long)k0 * N + (long long)a * NX;
        const float2* h1 = hh4 + (long long)(k1 < m ? k1 : k0) * N + (long long)a * NX;
        // partner row: the other group of this item, or this group for a in {0, NY/2}
        const float2* pbuf = (a == 0 || 2 * a == NY) ? b0 : pb0;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int cb = j + r * T;
            float2 X0, X1;
            split_dc_nyq(v[r], pbuf[padi(l1_partner_col(a, cb, NX))], X0, X1);
            acc[r] = cfma(__ldg(&h0[cb]), X0, acc[r]);
            if (k1 < m) acc[r] = cfma(__ldg(&h1[cb]), X1, acc[r]);
        }
    }
    fft<NX, true>(acc, j, b0, b1, tw);
    const bool store = active && (side == 0 || a != a0);
    if (store) {
        float2* Ar = A + (long long)b * N + (long long)a * NX;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int cc = j + r * T;
            Ar[cc] = cmulc(acc[r], __ldg(&twN[(long long)cc * a]));
        }
    }
}

// K3.  Grid (batch, NX / C).  y[b][c + NX r] = Re(column IFFT of A[b][.][c])[r] * scale.
template <int NY>
__global__ void __launch_bounds__(ColCfg<NY>::NT)
k4_cols_inv(const float2* __restrict__ A, int NX, float* __restrict__ y, float scale,
            const float2* __restrict__ tw) {
    using CC = ColCfg<NY>;
    constexpr int T = CC::T;
    constexpr int C = CC::C;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % C;
    const int j = threadIdx.x / C;
    float2* b0 = smem + c * CC::CS;
    float2* b1 = b0 + pad_len(NY);
    const int b = blockIdx.x;
    const int col = blockIdx.y * C + c;
    const bool cv = col < NX;
    const long long N = (long long)NY * NX;
    const float2* Ab = A + (long long)b * N;
    float2 v[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r)
        v[r] = cv ? __ldg(&Ab[(long long)(j + r * T) * NX + col]) : make_float2(0.f, 0.f);
    fft<NY, true, kColLayout>(v, j, b0, b1, tw);
    if (cv) {
        float* yb = y + (long long)b * N;
#pragma unroll
        for (int r = 0; r < kR; ++r) yb[(long long)(j + r * T) * NX + col] = v[r].x * scale;
    }
}

// K2'.  Grid (ceil(NY / (2 ITEMS)), batch): one row per group.  Row FFT of
// V once; per pair the product with conj(hhat_{2p}) + i conj(hhat_{2p+1}),
// row IFFT, conjugate twiddle, store Q[(b * npairs + p)][a][c].
template <int NX>
__global__ void __launch_bounds__(L1Rows<NX>::NT)
k4_rows_adj(const float2* __restrict__ V, int npairs, const float2* __restrict__ hh4, int m, int NY,
            const float2* __restrict__ twN, float2* __restrict__ Q, const float2* __restrict__ tw) {
    using L = L1Rows<NX>;
    constexpr int T = L::T;
    extern __shared__ float2 smem[];
    const int grp = threadIdx.x / T;
    const int j = threadIdx.x - grp * T;
    float2* b0 = smem + grp * fft_region(NX);
    float2* b1 = b0 + pad_len(NX);
    const int a0 = blockIdx.x * (2 * L::ITEMS) + grp;
    const bool active = a0 < NY;
    const int a = active ? a0 : 0;
    const int b = blockIdx.y;
    const long long N = (long long)NY * NX;
    float2 vv[kR];
    const float2* Vr = V + (long long)b * N + (long long)a * NX;
#pragma unroll
    for (int r = 0; r < kR; ++r) vv[r] = __ldg(&Vr[j + r * T]);
    fft<NX, false>(vv, j, b0, b1, tw);
    for (int p = 0; p < npairs; ++p) {
        const int k0 = 2 * p, k1 = 2 * p + 1;
        const float2* h0 = hh4 + (long long)k0 * N + (long long)a * NX;
        const float2* h1 = hh4 + (long long)(k1 < m ? k1 : k0) * N + (long long)a * NX;
        float2 q[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int cb = j + r * T;
            float2 t = cmulc(vv[r], __ldg(&h0[cb]));
            if (k1 < m) {
                const float2 s = cmulc(vv[r], __ldg(&h1[cb]));
                t.x -= s.y;
                t.y += s.x;
            }
            q[r] = t;
        }
        fft<NX, true>(q, j, b0, b1, tw);
        if (active) {
            float2* Qr = Q + ((long long)b * npairs + p) * N + (long long)a * NX;
#pragma unroll
            for (int r = 0; r < kR; ++r) {
                const int cc = j + r * T;
                Qr[cc] = cmulc(q[r], __ldg(&twN[(long long)cc * a]));
            }
        }
    }
}

// K3'.  Grid (batch, NX / C).  x[b][c + NX r] = scale * sum_p (w_{2p} Re + w_{2p+1} Im)
// of the column IFFT of Q[(b * npairs + p)][.][c].
template <int NY>
__global__ void __launch_bounds__(ColCfg<NY>::NT)
k4_cols_adj(const float2* __restrict__ Q, int npairs, const float* __restrict__ w, int m, int NX,
            float* __restrict__ x, float scale, const float2* __restrict__ tw) {
    using CC = ColCfg<NY>;
    constexpr int T = CC::T;
    constexpr int C = CC::C;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % C;
    const int j = threadIdx.x / C;
    float2* b0 = smem + c * CC::CS;
    float2* b1 = b0 + pad_len(NY);
    const int b = blockIdx.x;
    const int col = blockIdx.y * C + c;
    const bool cv = col < NX;
    const long long N = (long long)NY * NX;
    float acc[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) acc[r] = 0.f;
    for (int p = 0; p < npairs; ++p) {
        const float2* Qp = Q + ((long long)b * npairs + p) * N;
        float2 v[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r)
            v[r] = cv ? __ldg(&Qp[(long long)(j + r * T) * NX + col]) : make_float2(0.f, 0.f);
        fft<NY, true, kColLayout>(v, j, b0, b1, tw);
        const int k0 = 2 * p, k1 = 2 * p + 1;
        if (cv) {
#pragma unroll
            for (int r = 0; r < kR; ++r) {
                const long long n = col + (long long)NX * (j + r * T);
                acc[r] = fmaf(__ldg(w + (long long)k0 * N + n), v[r].x, acc[r]);
                if (k1 < m) acc[r] = fmaf(__ldg(w + (long long)k1 * N + n), v[r].y, acc[r]);
            }
        }
    }
    if (cv) {
        float* xb = x + (long long)b * N;
#pragma unroll
        for (int r = 0; r < kR; ++r) xb[(long long)(j + r * T) * NX + col] = acc[r] * scale;
    }
}

// Plan: the separated spectra of h_{2p}, h_{2p+1} in the four-step order,
// hh4[k][a][col].  Grid (ceil((NY/2 + 1) / ITEMS), npairs).
template <int NX>
__global__ void __launch_bounds__(L1Rows<NX>::NT)
k4_rows_spec(const float2* __restrict__ G, int npairs, int m, int NY, float2* __restrict__ hh4,
             const float2* __restrict__ tw) {
    using L = L1Rows<NX>;
    constexpr int T = L::T;
    extern __shared__ float2 smem[];
    const int grp = threadIdx.x / T;
    const int j = threadIdx.x - grp * T;
    const int item = grp >> 1, side = grp & 1;
    float2* b0 = smem + grp * fft_region(NX);
    float2* b1 = b0 + pad_len(NX);
    float2* pb0 = smem + (grp ^ 1) * fft_region(NX);
    const int a0 = blockIdx.x * L::ITEMS + item;
    const bool active = a0 <= NY / 2;
    const int a = side == 0 ? (active ? a0 : 0) : ((NY - (active ? a0 : 0)) & (NY - 1));
    const int p = blockIdx.y;
    const long long N = (long long)NY * NX;
    const float2* Gr = G + (long long)p * N + (long long)a * NX;
    float2 v[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) v[r] = __ldg(&Gr[j + r * T]);
    fft<NX, false>(v, j, b0, b1, tw);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kR; ++r) b0[padi(j + r * T)] = v[r];
    __syncthreads();
    const float2* pbuf = (a == 0 || 2 * a == NY) ? b0 : pb0;
    const int k0 = 2 * p, k1 = 2 * p + 1;
    const bool store = active && (side == 0 || a != a0);
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int cb = j + r * T;
        float2 X0, X1;
        split_dc_nyq(v[r], pbuf[padi(l1_partner_col(a, cb, NX))], X0, X1);
        if (store) {
            hh4[(long long)k0 * N + (long long)a * NX + cb] = X0;
            if (k1 < m) hh4[(long long)k1 * N + (long long)a * NX + cb] = X1;
        }
    }
}

}  // namespace pce
