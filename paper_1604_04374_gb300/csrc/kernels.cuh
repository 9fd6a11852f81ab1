// kernels.cuh -- CUDA kernels of the convolution-product expansion (Eq. 1.4).
//
// 2D forward  y_b = C2R( sum_k hhat_k . R2C(w_k . u_b) ) / P, three passes:
//   F1 k_rows_r2c<WINDOW=true>: for every active row of w_k's support box,
//      w_k . u_b restricted to the box columns, R2C along x (two real rows
//      per complex FFT), written to the intermediate Z[b][k][row in box].
//   F2 k_cols_fwd: per column of the half spectrum: for each k the column
//      FFT of Z_{b,k} (input nonzero only on the box rows), times hhat_k,
//      accumulated in registers; then one inverse column FFT.
//   F3 k_rows_c2r: C2R along x, times 1/P.
// 2D adjoint  x_b = sum_k w_k . C2R( conj(hhat_k) . R2C(v_b) ) / P:
//   G1 k_rows_r2c<WINDOW=false>, G2 k_cols_adj (column FFT once, then per k
//   the product with conj(hhat_k) and an inverse column FFT whose output is
//   kept only on w_k's box rows), G3 k_rows_adj (per row: C2R of each term
//   whose box holds the row, times w_k, accumulated in registers).
// 1D (N <= 8192): one CTA per right-hand side does all of it (k_fwd_1d,
//   k_adj_1d).
//
// Half-spectrum layout ("packed"): a real row of NX samples has its R2C
// spectrum stored as NX/2 complex values, slot 0 holding (X[0], X[NX/2]) (both
// real) and slot f = X[f] for 0 < f < NX/2.  In 2D the column FFT of slot 0
// therefore transforms DC + i * Nyquist; the two are separated with
// A[f] = (Z[f] + conj Z[-f]) / 2, B[f] = (Z[f] - conj Z[-f]) / (2i).
#pragma once

#include "fft.cuh"

namespace pce {

struct Box {          // periodic support box of w_k and its compacted copy
    int r0, nr;       // first row, number of rows (rows r0 .. r0+nr-1 mod Ny)
    int c0, nc;       // first column, number of columns (mod Nx)
    long long woff;   // offset of the [nr][ldw] box copy in the window buffer
    int ldw;          // row stride of the box copy
    int pad_;
};

// Sectioned apply (section.cuh): a term's input and output windows, as box
// offsets relative to the box origin (r0, c0).
struct SecGeom {
    int r0, c0;             // box origin in the grid
    int in_lo_r, in_rows;   // input rows: box offsets in_lo_r .. in_lo_r + in_rows - 1
    int in_lo_c, in_hi_c;   // input columns: box offsets in_lo_c .. in_hi_c
    int out_lo_r, out_rows;
    int out_lo_c, out_hi_c;
    long long woff;         // window box copy [nr][ldw] (the box of w_k), at the section's first column
    int ldw, k;             // k: the term whose section spectrum the section uses
};

// Separable windows w_k = wy_k (x) wx_k: terms sharing the column factor wx
// share one slot of row spectra R_j = R2C_x(wx_j . u) (rows of the slot box).
struct SepTerms {
    const float* wrow = nullptr;   // [m][Ny] row factors wy_k
    const int* kslot = nullptr;    // [m] slot of every term
    const int* korder = nullptr;   // [nterms] the terms to run, grouped by slot
    int nterms = 0;
    const int* kq0 = nullptr;      // [m] pruned column kernels: wy_k's rows lie in [32 kq0, 32 kq0 + 512)
    // slot-by-slot schedule of the tensor-memory column kernels: the terms
    // korder[t0 .. t1) of this pass (t1 < 0: all) and the pass's mode bits
    int t0 = 0, t1 = -1, mode = 0;
};
// mode bits (forward): the accumulator starts from A (frequency domain) / the
// pass ends with the inverse FFT (else A receives the frequency-domain sum)
constexpr int kSepLoadAcc = 1, kSepFinal = 2;
// mode bits (adjoint): V already holds its column spectrum / store the column
// spectrum back into V for later passes
constexpr int kSepSpecIn = 4, kSepSpecOut = 8;

// i mod n for a power of two n (two's complement: also for negative i)
__device__ __forceinline__ int wrap(int i, int n) { return i & (n - 1); }

// ---------------------------------------------------------------- rows R2C
// Real rows -> packed half spectra, two rows per complex FFT.
// WINDOW: item = (k, p) -> box rows 2p, 2p+1 of w_k (global rows r0+2p, r0+2p+1),
//         multiplied by the box copy of w_k, output rows 2p, 2p+1 of dst[b][k].
// !WINDOW: item = p -> rows 2p, 2p+1 (< nrows), output rows 2p, 2p+1 of dst[b].
// Each slot handles kRowIters items one after the other; the inputs of the
// next item are loaded before the FFT of the current one.
constexpr int kRowIters = 1;

template <typename WT>
struct RowItem {
    int k, la, lb;
    bool va, vb;
    const float* sa;
    const float* sb;
    const WT* wa;   // window row of la (WINDOW), nullptr otherwise
    const WT* wb;
    int c0, nc;
};

template <int NX, bool WINDOW, typename WT>
__device__ __forceinline__ RowItem<WT> row_item(int item, int nitems, const float* __restrict__ src, int nrows,
                                                const WT* __restrict__ wbox, const Box* __restrict__ box,
                                                const int2* __restrict__ items) {
    RowItem<WT> it;
    const bool active = item < nitems;
    if (WINDOW) {
        const int2 kp = active ? items[item] : make_int2(0, 0);
        const Box bx = box[kp.x];
        it.k = kp.x;
        it.la = 2 * kp.y;
        it.lb = it.la + 1;
        it.va = active && it.la < bx.nr;
        it.vb = active && it.lb < bx.nr;
        it.sa = src + (long long)wrap(bx.r0 + it.la, nrows) * NX;
        it.sb = src + (long long)wrap(bx.r0 + it.lb, nrows) * NX;
        it.wa = wbox + bx.woff + (long long)it.la * bx.ldw;
        it.wb = wbox + bx.woff + (long long)it.lb * bx.ldw;
        it.c0 = bx.c0;
        it.nc = bx.nc;
    } else {
        it.k = 0;
        it.la = 2 * item;
        it.lb = it.la + 1;
        it.va = active && it.la < nrows;
        it.vb = active && it.lb < nrows;
        it.sa = src + (long long)(it.va ? it.la : 0) * NX;
        it.sb = src + (long long)(it.vb ? it.lb : 0) * NX;
        it.wa = it.wb = nullptr;
        it.c0 = 0;
        it.nc = NX;
    }
    return it;
}

template <int NX, bool WINDOW, typename WT>
__device__ __forceinline__ void row_load(float2 (&v)[kR], const RowItem<WT>& it, int j) {
    constexpr int T = NX / kR;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int n = j + r * T;
        float xa = 0.f, xb = 0.f;
        if (WINDOW) {
            const int cc = wrap(n - it.c0, NX);
            if (cc < it.nc) {
                if (it.va) xa = ldw(it.wa + cc) * __ldg(it.sa + n);
                if (it.vb) xb = ldw(it.wb + cc) * __ldg(it.sb + n);
            }
        } else {
            if (it.va) xa = __ldg(it.sa + n);
            if (it.vb) xb = __ldg(it.sb + n);
        }
        v[r] = make_float2(xa, xb);
    }
}

template <int NX, bool WINDOW, typename WT = float>
__global__ void __launch_bounds__(256)
k_rows_r2c(const float* __restrict__ src, long long src_bstride, int nrows,
           const WT* __restrict__ wbox, const Box* __restrict__ box,
           const int2* __restrict__ items, int nitems,
           float2* __restrict__ dst, long long dst_bstride, long long dst_kstride,
           const float2* __restrict__ tw) {
    constexpr int T = NX / kR;
    constexpr int FPC = 256 / T;
    constexpr int NXh = NX / 2;
    __shared__ float2 sbuf[FPC * fft_region(NX)];
    const int slot = threadIdx.x / T;
    const int j = threadIdx.x - slot * T;
    float2* b0 = sbuf + slot * fft_region(NX);
    float2* b1 = b0 + pad_len(NX);
    const int b = blockIdx.y;
    const float* srcb = src + b * src_bstride;
    const int first = blockIdx.x * kRowIters * FPC + slot;

    RowItem<WT> cur = row_item<NX, WINDOW, WT>(first, nitems, srcb, nrows, wbox, box, items);
    float2 v[kR];
    row_load<NX, WINDOW, WT>(v, cur, j);
    for (int it = 0; it < kRowIters; ++it) {
        RowItem<WT> nxt;
        float2 vn[kR];
        const bool more = it + 1 < kRowIters;
        if (more) {
            nxt = row_item<NX, WINDOW, WT>(first + (it + 1) * FPC, nitems, srcb, nrows, wbox, box, items);
            row_load<NX, WINDOW, WT>(vn, nxt, j);
        }
        fft<NX, false>(v, j, b0, b1, tw);

        // split the spectra of the two real rows
        float2* xs = b0;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kR; ++r) xs[padi(j + r * T)] = v[r];
        __syncthreads();
        float2* da = dst + b * dst_bstride + cur.k * dst_kstride + (long long)cur.la * NXh;
        float2* db = dst + b * dst_bstride + cur.k * dst_kstride + (long long)cur.lb * NXh;
#pragma unroll
        for (int r = 0; r < kR / 2; ++r) {
            const int f = j + r * T;
            float2 A, B;
            if (f == 0) {
                A = make_float2(v[0].x, v[kR / 2].x);
                B = make_float2(v[0].y, v[kR / 2].y);
            } else {
                const float2 z = v[r];
                const float2 zm = xs[padi(NX - f)];
                A = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
                B = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
            }
            if (cur.va) da[f] = A;
            if (cur.vb) db[f] = B;
        }
        if (more) {
            cur = nxt;
#pragma unroll
            for (int r = 0; r < kR; ++r) v[r] = vn[r];
        }
    }
}

// F1 by row pairs: the two input rows are loaded once, then windowed and
// transformed for every term (or slot) whose box holds them -- the CSR lists
// kptr/klist of the adjoint row pass -- writing Z[b][k] rows (row - r0 of the
// box), as k_rows_r2c<NX, true> does item by item.  The separable plans'
// slots share every row, so the loads of u are amortised over the slots
// instead of repeated per slot.  Grid (ceil(npairs / FPC), batch), 256
// threads, 64 registers (4 CTAs per SM).
template <int NX, typename WT = float>
__global__ void __launch_bounds__(256, 4)
k_rows_r2c_pairs(const float* __restrict__ src, long long src_bstride, int nrows, const WT* __restrict__ wbox,
                 const Box* __restrict__ box, const int* __restrict__ kptr, const int* __restrict__ klist,
                 float2* __restrict__ dst, long long dst_bstride, long long dst_kstride,
                 const float2* __restrict__ tw) {
    constexpr int T = NX / kR;
    constexpr int FPC = 256 / T;
    constexpr int NXh = NX / 2;
    __shared__ float2 sbuf[FPC * fft_region(NX)];
    const int slot = threadIdx.x / T;
    const int j = threadIdx.x - slot * T;
    float2* b0 = sbuf + slot * fft_region(NX);
    float2* b1 = b0 + pad_len(NX);
    const int npairs = (nrows + 1) / 2;
    const int p = blockIdx.x * FPC + slot;
    const int b = blockIdx.y;
    const bool pv = p < npairs;
    const int ga = 2 * p, gb = ga + 1;
    const bool hb = pv && gb < nrows;
    // uniform trip count over the CTA's row pairs (the FFT has CTA barriers)
    int nk = 0;
    for (int s2 = 0; s2 < FPC; ++s2) {
        const int ps = blockIdx.x * FPC + s2;
        if (ps < npairs) nk = max(nk, __ldg(&kptr[ps + 1]) - __ldg(&kptr[ps]));
    }
    const int kbeg = pv ? __ldg(&kptr[p]) : 0;
    const int kcnt = pv ? __ldg(&kptr[p + 1]) - kbeg : 0;
    float ua[kR], ub[kR];
    {
        const float* sa = src + b * src_bstride + (long long)(pv ? ga : 0) * NX;
        const float* sb = src + b * src_bstride + (long long)(hb ? gb : 0) * NX;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            ua[r] = pv && kcnt > 0 ? __ldg(sa + j + r * T) : 0.f;
            ub[r] = hb && kcnt > 0 ? __ldg(sb + j + r * T) : 0.f;
        }
    }
    for (int t = 0; t < nk; ++t) {
        const bool act = t < kcnt;
        const int k = act ? __ldg(&klist[kbeg + t]) : 0;
        const Box bx = box[k];
        const int la = wrap(ga - bx.r0, nrows), lb = wrap(gb - bx.r0, nrows);
        const bool va = act && la < bx.nr;
        const bool vb = act && hb && lb < bx.nr;
        const WT* wa = wbox + bx.woff + (long long)(va ? la : 0) * bx.ldw;
        const WT* wb = wbox + bx.woff + (long long)(vb ? lb : 0) * bx.ldw;
        float2 v[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int n = j + r * T;
            const int cc = wrap(n - bx.c0, NX);
            const bool in = cc < bx.nc;
            v[r] = make_float2(va && in ? ldw(wa + cc) * ua[r] : 0.f, vb && in ? ldw(wb + cc) * ub[r] : 0.f);
        }
        fft<NX, false>(v, j, b0, b1, tw);
        // split the spectra of the two real rows
        float2* xs = b0;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kR; ++r) xs[padi(j + r * T)] = v[r];
        __syncthreads();
        float2* da = dst + b * dst_bstride + k * dst_kstride + (long long)la * NXh;
        float2* db = dst + b * dst_bstride + k * dst_kstride + (long long)lb * NXh;
#pragma unroll
        for (int r = 0; r < kR / 2; ++r) {
            const int f = j + r * T;
            float2 A, B;
            if (f == 0) {
                A = make_float2(v[0].x, v[kR / 2].x);
                B = make_float2(v[0].y, v[kR / 2].y);
            } else {
                const float2 z = v[r];
                const float2 zm = xs[padi(NX - f)];
                A = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
                B = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
            }
            if (va) da[f] = A;
            if (vb) db[f] = B;
        }
    }
}

// ---------------------------------------------------------------- rows C2R
// Packed half spectra -> real rows (two rows per complex inverse FFT), times scale.
// Value at frequency f in [0, NX) of the spectrum whose packed half is p
// (Hermitian extension; DC and Nyquist are the real parts kept in slot 0).
template <int NX>
__device__ __forceinline__ float2 load_half(const float2* p, int f) {
    constexpr int NXh = NX / 2;
    if (f == 0) return make_float2(p[0].x, 0.f);
    if (f == NXh) return make_float2(p[0].y, 0.f);
    if (f < NXh) return p[f];
    return cconj(p[NX - f]);
}
// The same from a stored spectrum (FP32, or FP16 times the term's scale s).
template <int NX, typename HT>
__device__ __forceinline__ float2 load_half_h(const HT* p, int f, float s) {
    constexpr int NXh = NX / 2;
    if (f == 0) return make_float2(ldh(&p[0], s).x, 0.f);
    if (f == NXh) return make_float2(ldh(&p[0], s).y, 0.f);
    if (f < NXh) return ldh(&p[f], s);
    return cconj(ldh(&p[NX - f], s));
}

template <int NX>
__global__ void __launch_bounds__(256)
k_rows_c2r(const float2* __restrict__ src, long long src_bstride, int nrows,
           float* __restrict__ dst, long long dst_bstride, float scale,
           const float2* __restrict__ tw) {
    constexpr int T = NX / kR;
    constexpr int FPC = 256 / T;
    constexpr int NXh = NX / 2;
    __shared__ float2 sbuf[FPC * fft_region(NX)];
    const int slot = threadIdx.x / T;
    const int j = threadIdx.x - slot * T;
    float2* b0 = sbuf + slot * fft_region(NX);
    float2* b1 = b0 + pad_len(NX);
    const int p = blockIdx.x * FPC + slot;
    const int b = blockIdx.y;
    const int la = 2 * p, lb = la + 1;
    const bool va = la < nrows, vb = lb < nrows;
    const float2* pa = src + b * src_bstride + (long long)(va ? la : 0) * NXh;
    const float2* pb = src + b * src_bstride + (long long)(vb ? lb : 0) * NXh;
    float2 v[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int f = j + r * T;
        const float2 xa = va ? load_half<NX>(pa, f) : make_float2(0.f, 0.f);
        const float2 xb = vb ? load_half<NX>(pb, f) : make_float2(0.f, 0.f);
        v[r] = make_float2(xa.x - xb.y, xa.y + xb.x);
    }
    fft<NX, true>(v, j, b0, b1, tw);
    float* ya = dst + b * dst_bstride + (long long)la * NX;
    float* yb = dst + b * dst_bstride + (long long)lb * NX;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int n = j + r * T;
        if (va) ya[n] = v[r].x * scale;
        if (vb) yb[n] = v[r].y * scale;
    }
}

// ------------------------------------------------------ rows C2R, adjoint G3
// Row pair (2p, 2p+1): x = sum over the terms k whose box holds the row of
// w_k . C2R(Q_{b,k}[row]), times scale.  Q rows are indexed inside the box.
// The next term's Q rows and window values are loaded before the inverse
// FFT of the current term.
template <typename WT>
struct AdjTerm {
    const float2* pa;
    const float2* pb;
    const WT* wa;
    const WT* wb;
    bool va, vb;
    int c0, nc;
};

template <int NX, typename WT>
__device__ __forceinline__ void adj_load(float2 (&v)[kR], float (&wa)[kR], float (&wb)[kR],
                                         const AdjTerm<WT>& q, int j) {
    constexpr int T = NX / kR;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int f = j + r * T;
        const float2 xa = q.va ? load_half<NX>(q.pa, f) : make_float2(0.f, 0.f);
        const float2 xb = q.vb ? load_half<NX>(q.pb, f) : make_float2(0.f, 0.f);
        v[r] = make_float2(xa.x - xb.y, xa.y + xb.x);
        const int cc = wrap(f - q.c0, NX);     // f doubles as the output column n = j + r*T
        const bool in = cc < q.nc;
        wa[r] = (q.va && in) ? ldw(q.wa + cc) : 0.f;
        wb[r] = (q.vb && in) ? ldw(q.wb + cc) : 0.f;
    }
}

// RV = 0: the next term's Q rows and window values are prefetched into
// registers during the current term's FFT (128 registers, 2 CTAs per SM);
// RV = 1: no prefetch, 80 registers, 3 CTAs per SM (more warps hide the
// loads instead).  The autotuner picks one per plan.
template <int NX, typename WT = float, int RV = 0>
__global__ void __launch_bounds__(256, RV == 1 ? 3 : 1)
k_rows_adj(const float2* __restrict__ Q, long long q_bstride, long long q_kstride, int nrows,
           const WT* __restrict__ wbox, const Box* __restrict__ box,
           const int* __restrict__ kptr, const int* __restrict__ klist,
           float* __restrict__ dst, long long dst_bstride, float scale,
           const float2* __restrict__ tw, int kmin, int kmax, int accumulate) {
    constexpr int T = NX / kR;
    constexpr int FPC = 256 / T;
    constexpr int NXh = NX / 2;
    __shared__ float2 sbuf[FPC * fft_region(NX)];
    const int slot = threadIdx.x / T;
    const int j = threadIdx.x - slot * T;
    float2* b0 = sbuf + slot * fft_region(NX);
    float2* b1 = b0 + pad_len(NX);
    const int npairs = (nrows + 1) / 2;
    const int p = blockIdx.x * FPC + slot;
    const int b = blockIdx.y;
    const bool pv = p < npairs;
    const int ga = 2 * p, gb = ga + 1;

    // the row pair's entries with kmin <= k < kmax (each list is sorted by k, so
    // they are contiguous); uniform trip count over the CTA's row pairs
    auto range = [&](int ps, int& beg, int& cnt) {
        int a = __ldg(&kptr[ps]), e = __ldg(&kptr[ps + 1]);
        while (a < e && __ldg(&klist[a]) < kmin) ++a;
        int z = a;
        while (z < e && __ldg(&klist[z]) < kmax) ++z;
        beg = a;
        cnt = z - a;
    };
    int nk = 0;
    for (int s = 0; s < FPC; ++s) {
        const int ps = blockIdx.x * FPC + s;
        if (ps < npairs) {
            int bs, cs;
            range(ps, bs, cs);
            nk = max(nk, cs);
        }
    }
    int kbeg = 0, kcnt = 0;
    if (pv) range(p, kbeg, kcnt);

    auto term = [&](int t) {
        AdjTerm<WT> q;
        const bool act = t < kcnt;
        const int k = act ? __ldg(&klist[kbeg + t]) : 0;
        const Box bx = box[k];
        const int la = wrap(ga - bx.r0, nrows);
        const int lb = wrap(gb - bx.r0, nrows);
        q.va = act && la < bx.nr;
        q.vb = act && gb < nrows && lb < bx.nr;
        q.pa = Q + b * q_bstride + k * q_kstride + (long long)(q.va ? la : 0) * NXh;
        q.pb = Q + b * q_bstride + k * q_kstride + (long long)(q.vb ? lb : 0) * NXh;
        q.wa = wbox + bx.woff + (long long)(q.va ? la : 0) * bx.ldw;
        q.wb = wbox + bx.woff + (long long)(q.vb ? lb : 0) * bx.ldw;
        q.c0 = bx.c0;
        q.nc = bx.nc;
        return q;
    };

    float2 acc[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) acc[r] = make_float2(0.f, 0.f);

    float2 v[kR];
    float wa[kR], wb[kR];
    if constexpr (RV == 1) {
        for (int t = 0; t < nk; ++t) {
            adj_load<NX, WT>(v, wa, wb, term(t), j);
            fft<NX, true>(v, j, b0, b1, tw);
#pragma unroll
            for (int r = 0; r < kR; ++r) {
                acc[r].x = fmaf(wa[r], v[r].x, acc[r].x);
                acc[r].y = fmaf(wb[r], v[r].y, acc[r].y);
            }
        }
    } else {
        if (nk > 0) adj_load<NX, WT>(v, wa, wb, term(0), j);
        for (int t = 0; t < nk; ++t) {
            float2 vn[kR];
            float wan[kR], wbn[kR];
            const bool more = t + 1 < nk;
            if (more) adj_load<NX, WT>(vn, wan, wbn, term(t + 1), j);
            fft<NX, true>(v, j, b0, b1, tw);
#pragma unroll
            for (int r = 0; r < kR; ++r) {
                acc[r].x = fmaf(wa[r], v[r].x, acc[r].x);
                acc[r].y = fmaf(wb[r], v[r].y, acc[r].y);
            }
            if (more) {
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    v[r] = vn[r];
                    wa[r] = wan[r];
                    wb[r] = wbn[r];
                }
            }
        }
    }
    float* xa = dst + b * dst_bstride + (long long)ga * NX;
    float* xb = dst + b * dst_bstride + (long long)gb * NX;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int n = j + r * T;
        if (accumulate) {   // a later pass of the slot-by-slot schedule adds its slots
            if (pv) xa[n] += acc[r].x * scale;
            if (pv && gb < nrows) xb[n] += acc[r].y * scale;
        } else {
            if (pv) xa[n] = acc[r].x * scale;
            if (pv && gb < nrows) xb[n] = acc[r].y * scale;
        }
    }
}

// ------------------------------------------------------------ column passes
// CTA = C columns x T threads; thread (j, c) = threadIdx (j * C + c), so a
// warp reads C consecutive columns of 8 rows (32-byte segments for C = 4).
// Each column owns two FFT buffers; consecutive columns' buffers are skewed
// by 4 float2 (32 bytes) so that the C columns of a warp fall on distinct
// shared-memory banks.
template <int NY>
struct ColCfg {
    static constexpr int T = NY / kR;
    static constexpr int C = (4 * T >= 128) ? (T >= 256 ? 2 : 4) : 128 / T;   // columns per CTA
    static constexpr int NT = T * C;                          // threads per CTA
    static constexpr int CS = fft_region(NY);                 // per-column region (float2)
    static constexpr int SMEM = (C * CS + pad_len(NY)) * (int)sizeof(float2);
};

// Separate the column FFT Z of (DC + i Nyquist) at frequency f.
__device__ __forceinline__ void split_dc_nyq(float2 z, float2 zm, float2& A, float2& B) {
    A = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
    B = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
}

template <int NY>
__device__ __forceinline__ void load_col(float2 (&v)[kR], const float2* __restrict__ Zk, const Box& bx,
                                         int j, int col, int nxh, bool cv) {
    constexpr int T = NY / kR;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int i = wrap(j + r * T - bx.r0, NY);
        v[r] = (cv && i < bx.nr) ? __ldg(&Zk[(long long)i * nxh + col]) : make_float2(0.f, 0.f);
    }
}

// F2: forward column pass.  Grid (batch, NXh / C): the right-hand sides of a
// column tile are neighbours in launch order and share hhat_k through L2.
// hh: [m][NY][NXh] (column 0 = DC column spectrum), hN: [m][NY] (Nyquist).
// The next term's Z column and this term's spectrum are loaded before the
// FFT so that their latency overlaps it.
template <int NY, typename HT = float2>
__global__ void __launch_bounds__(ColCfg<NY>::NT)
k_cols_fwd(const float2* __restrict__ Z, long long z_bstride, long long z_kstride,
           const HT* __restrict__ hh, const HT* __restrict__ hN, const float* __restrict__ hscale, int m,
           const Box* __restrict__ box, int NXh,
           float2* __restrict__ A, long long a_bstride, const float2* __restrict__ tw) {
    using CC = ColCfg<NY>;
    constexpr int T = CC::T;
    constexpr int C = CC::C;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % C;
    const int j = threadIdx.x / C;
    float2* b0 = smem + c * CC::CS;
    float2* b1 = b0 + pad_len(NY);
    float2* xbuf = smem + C * CC::CS;
    const int b = blockIdx.x;
    const int tile = blockIdx.y;
    const int col = tile * C + c;
    const bool cv = col < NXh;
    const bool tile0 = tile == 0;
    const bool dcn = tile0 && c == 0;
    const float2* Zb = Z + b * z_bstride;

    float2 acc[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) acc[r] = make_float2(0.f, 0.f);

    // first term with a nonempty box
    int k = 0;
    while (k < m && box[k].nr == 0) ++k;
    if (k >= m) {
        // every window is zero: the output spectrum is zero
        fft<NY, true, kColLayout>(acc, j, b0, b1, tw);
        if (cv) {
            float2* Ab = A + b * a_bstride;
#pragma unroll
            for (int r = 0; r < kR; ++r) Ab[(long long)(j + r * T) * NXh + col] = acc[r];
        }
        return;
    }
    Box bx = box[k];
    float2 v[kR];
    load_col<NY>(v, Zb + k * z_kstride, bx, j, col, NXh, cv);

    while (k < m) {
        // next term with a nonempty box
        int kn = k + 1;
        while (kn < m && box[kn].nr == 0) ++kn;
        // spectrum of term k at this thread's frequencies
        const HT* hk = hh + (long long)k * NY * NXh;
        const float sk = hscale_of<HT>(hscale, k);
        float2 hv[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r)
            hv[r] = cv ? ldh(&hk[(long long)(j + r * T) * NXh + col], sk) : make_float2(0.f, 0.f);
        // Z column of the next term
        float2 zn[kR];
        Box bn = bx;
        if (kn < m) {
            bn = box[kn];
            load_col<NY>(zn, Zb + kn * z_kstride, bn, j, col, NXh, cv);
        }
        fft<NY, false, kColLayout>(v, j, b0, b1, tw);
        if (tile0) {
            if (dcn) {
#pragma unroll
                for (int r = 0; r < kR; ++r) xbuf[padi(j + r * T)] = v[r];
            }
            __syncthreads();
        }
        if (dcn) {
#pragma unroll
            for (int r = 0; r < kR; ++r) {
                const int f = j + r * T;
                float2 a, bb;
                split_dc_nyq(v[r], xbuf[padi((NY - f) & (NY - 1))], a, bb);
                acc[r] = cfma(hv[r], a, acc[r]);
                const float2 t = cmul(ldh(&hN[(long long)k * NY + f], sk), bb);
                acc[r].x -= t.y;
                acc[r].y += t.x;
            }
        } else {
#pragma unroll
            for (int r = 0; r < kR; ++r) acc[r] = cfma(hv[r], v[r], acc[r]);
        }
        if (kn < m) {
#pragma unroll
            for (int r = 0; r < kR; ++r) v[r] = zn[r];
        }
        k = kn;
        bx = bn;
    }
    fft<NY, true, kColLayout>(acc, j, b0, b1, tw);
    if (cv) {
        float2* Ab = A + b * a_bstride;
#pragma unroll
        for (int r = 0; r < kR; ++r) Ab[(long long)(j + r * T) * NXh + col] = acc[r];
    }
}

// G1b + G2: adjoint column pass.  Column FFT of V once; per k the product
// with conj(hhat_k), an inverse column FFT, and a store of the box rows only
// (FULL: of every row, Q[b][k][NY][NXh], for the window gradient).
// Grid (batch, NXh / C).  The next term's spectrum is loaded before the
// current inverse FFT.
template <int NY, bool FULL, typename HT = float2>
__global__ void __launch_bounds__(ColCfg<NY>::NT)
k_cols_adj(const float2* __restrict__ V, long long v_bstride,
           const HT* __restrict__ hh, const HT* __restrict__ hN, const float* __restrict__ hscale, int m,
           const Box* __restrict__ box, int NXh,
           float2* __restrict__ Q, long long q_bstride, long long q_kstride,
           const float2* __restrict__ tw) {
    using CC = ColCfg<NY>;
    constexpr int T = CC::T;
    constexpr int C = CC::C;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % C;
    const int j = threadIdx.x / C;
    float2* b0 = smem + c * CC::CS;
    float2* b1 = b0 + pad_len(NY);
    float2* xbuf = smem + C * CC::CS;
    const int b = blockIdx.x;
    const int tile = blockIdx.y;
    const int col = tile * C + c;
    const bool cv = col < NXh;
    const bool tile0 = tile == 0;
    const bool dcn = tile0 && c == 0;

    float2 vv[kR];
    const float2* Vb = V + b * v_bstride;
#pragma unroll
    for (int r = 0; r < kR; ++r)
        vv[r] = cv ? __ldg(&Vb[(long long)(j + r * T) * NXh + col]) : make_float2(0.f, 0.f);
    int k = 0;
    while (k < m && !FULL && box[k].nr == 0) ++k;
    float2 hv[kR];
    if (k < m) {
        const HT* hk = hh + (long long)k * NY * NXh;
        const float sk = hscale_of<HT>(hscale, k);
#pragma unroll
        for (int r = 0; r < kR; ++r)
            hv[r] = cv ? ldh(&hk[(long long)(j + r * T) * NXh + col], sk) : make_float2(0.f, 0.f);
    }
    fft<NY, false, kColLayout>(vv, j, b0, b1, tw);
    if (tile0) {
        if (dcn) {
#pragma unroll
            for (int r = 0; r < kR; ++r) xbuf[padi(j + r * T)] = vv[r];
        }
        __syncthreads();
    }
    while (k < m) {
        int kn = k + 1;
        while (kn < m && !FULL && box[kn].nr == 0) ++kn;
        const Box bx = box[k];
        float2 p[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int f = j + r * T;
            if (dcn) {
                float2 a, bb;
                split_dc_nyq(vv[r], xbuf[padi((NY - f) & (NY - 1))], a, bb);
                float2 t = cmulc(a, hv[r]);
                const float2 s = cmulc(bb, ldh(&hN[(long long)k * NY + f], hscale_of<HT>(hscale, k)));
                t.x -= s.y;
                t.y += s.x;
                p[r] = t;
            } else {
                p[r] = cmulc(vv[r], hv[r]);
            }
        }
        if (kn < m) {
            const HT* hk = hh + (long long)kn * NY * NXh;
            const float sk = hscale_of<HT>(hscale, kn);
#pragma unroll
            for (int r = 0; r < kR; ++r)
                hv[r] = cv ? ldh(&hk[(long long)(j + r * T) * NXh + col], sk) : make_float2(0.f, 0.f);
        }
        fft<NY, true, kColLayout>(p, j, b0, b1, tw);
        if (cv) {
            float2* Qk = Q + b * q_bstride + k * q_kstride;
#pragma unroll
            for (int r = 0; r < kR; ++r) {
                if (FULL) {
                    Qk[(long long)(j + r * T) * NXh + col] = p[r];
                } else {
                    const int i = wrap(j + r * T - bx.r0, NY);
                    if (i < bx.nr) Qk[(long long)i * NXh + col] = p[r];
                }
            }
        }
        k = kn;
    }
}

// Plan: column FFT of the row spectra of h_k -> hh (column 0 = DC column
// spectrum) and hN (Nyquist column spectrum).  Grid (m, NXh / C).
template <int NY>
__global__ void __launch_bounds__(ColCfg<NY>::NT)
k_cols_spec(const float2* __restrict__ S, int NXh, float2* __restrict__ hh,
            float2* __restrict__ hN, const float2* __restrict__ tw) {
    using CC = ColCfg<NY>;
    constexpr int T = CC::T;
    constexpr int C = CC::C;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % C;
    const int j = threadIdx.x / C;
    float2* b0 = smem + c * CC::CS;
    float2* b1 = b0 + pad_len(NY);
    float2* xbuf = smem + C * CC::CS;
    const int k = blockIdx.x;
    const int tile = blockIdx.y;
    const int col = tile * C + c;
    const bool cv = col < NXh;
    const bool tile0 = tile == 0;
    const bool dcn = tile0 && c == 0;
    const float2* Sk = S + (long long)k * NY * NXh;
    float2 v[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r)
        v[r] = cv ? __ldg(&Sk[(long long)(j + r * T) * NXh + col]) : make_float2(0.f, 0.f);
    fft<NY, false, kColLayout>(v, j, b0, b1, tw);
    if (tile0) {
        if (dcn) {
#pragma unroll
            for (int r = 0; r < kR; ++r) xbuf[padi(j + r * T)] = v[r];
        }
        __syncthreads();
    }
    float2* hk = hh + (long long)k * NY * NXh;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int f = j + r * T;
        if (dcn) {
            float2 a, bb;
            split_dc_nyq(v[r], xbuf[padi((NY - f) & (NY - 1))], a, bb);
            hk[(long long)f * NXh] = a;
            hN[(long long)k * NY + f] = bb;
        } else if (cv) {
            hk[(long long)f * NXh + col] = v[r];
        }
    }
}

// ------------------------------------------- plain unfused per-term path
// The comparator the fused kernels are measured against: for every term a
// window kernel, a full 2D R2C (row pass + column pass), and a spectral
// multiply-accumulate, each through global memory, then one inverse.

// Inverse column FFT from the [nb][ny][nxh] + Nyquist layout to packed row
// spectra A[nb][ny][nxh] (column 0 = IFFT(DC + i Nyquist)).  Grid (nb, NXh / C).
template <int NY>
__global__ void __launch_bounds__(ColCfg<NY>::NT)
k_plain_cols_inv(const float2* __restrict__ acc, const float2* __restrict__ accN, int NXh,
                 float2* __restrict__ A, const float2* __restrict__ tw) {
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
    const bool cv = col < NXh;
    const float2* ab = acc + (long long)b * NY * NXh;
    float2 v[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int f = j + r * T;
        float2 x = cv ? ab[(long long)f * NXh + col] : make_float2(0.f, 0.f);
        if (col == 0) {
            const float2 n = accN[(long long)b * NY + f];
            x.x -= n.y;
            x.y += n.x;
        }
        v[r] = x;
    }
    fft<NY, true, kColLayout>(v, j, b0, b1, tw);
    if (cv) {
        float2* Ab = A + (long long)b * NY * NXh;
#pragma unroll
        for (int r = 0; r < kR; ++r) Ab[(long long)(j + r * T) * NXh + col] = v[r];
    }
}

// ------------------------------------------------------------- gradients
// Backward of L(y), y = C2R( sum_k hhat_k . R2C(w_k . u) ), given r = dL/dy.
// With R_b = R2C(r_b) and X_{b,k} = R2C(w_k . u_b) (recomputed, not stored):
//   dL/dhhat_k = sum_b (c_f / P) R_b . conj(X_{b,k})   (c_f = 2 on the interior
//                columns of the half spectrum, 1 on DC and Nyquist; the
//                convention dL/dRe + i dL/dIm)
//   dL/dw_k    = sum_b u_b . C2R( conj(hhat_k) . R_b ) / P
//   dL/du_b    = H_m^* r_b (the adjoint apply).

// dhhat: grid (m, NXh / C).  Z: forward row spectra [nb][m][nr][NXh];
// Rh/RhN: column spectra of r in the kernels' layout.  Output natural
// [m][NY][NXh+1] complex; accumulate adds to it.
template <int NY>
__global__ void __launch_bounds__(ColCfg<NY>::NT)
k_cols_grad_h(const float2* __restrict__ Z, long long z_bstride, long long z_kstride, int nb,
              const float2* __restrict__ Rh, const float2* __restrict__ RhN,
              const Box* __restrict__ box, int NXh, float2* __restrict__ dhh, float scale,
              int accumulate, const float2* __restrict__ tw) {
    using CC = ColCfg<NY>;
    constexpr int T = CC::T;
    constexpr int C = CC::C;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % C;
    const int j = threadIdx.x / C;
    float2* b0 = smem + c * CC::CS;
    float2* b1 = b0 + pad_len(NY);
    float2* xbuf = smem + C * CC::CS;
    const int k = blockIdx.x;
    const int tile = blockIdx.y;
    const int col = tile * C + c;
    const bool cv = col < NXh;
    const bool tile0 = tile == 0;
    const bool dcn = tile0 && c == 0;
    const Box bx = box[k];
    float2 acc[kR], accN[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) acc[r] = accN[r] = make_float2(0.f, 0.f);
    if (bx.nr > 0) {
        float2 v[kR];
        load_col<NY>(v, Z + k * z_kstride, bx, j, col, NXh, cv);
        for (int b = 0; b < nb; ++b) {
            const bool more = b + 1 < nb;
            float2 vn[kR], rv[kR];
            if (more) load_col<NY>(vn, Z + (b + 1) * z_bstride + k * z_kstride, bx, j, col, NXh, cv);
            const float2* Rb = Rh + (long long)b * NY * NXh;
#pragma unroll
            for (int r = 0; r < kR; ++r)
                rv[r] = cv ? __ldg(&Rb[(long long)(j + r * T) * NXh + col]) : make_float2(0.f, 0.f);
            fft<NY, false, kColLayout>(v, j, b0, b1, tw);
            if (tile0) {
                if (dcn) {
#pragma unroll
                    for (int r = 0; r < kR; ++r) xbuf[padi(j + r * T)] = v[r];
                }
                __syncthreads();
            }
            if (dcn) {
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    const int f = j + r * T;
                    float2 a, bb;
                    split_dc_nyq(v[r], xbuf[padi((NY - f) & (NY - 1))], a, bb);
                    acc[r] = cfmac(a, rv[r], acc[r]);
                    accN[r] = cfmac(bb, __ldg(&RhN[(long long)b * NY + f]), accN[r]);
                }
            } else {
#pragma unroll
                for (int r = 0; r < kR; ++r) acc[r] = cfmac(v[r], rv[r], acc[r]);
            }
            if (more) {
#pragma unroll
                for (int r = 0; r < kR; ++r) v[r] = vn[r];
            }
        }
    }
    float2* dk = dhh + (long long)k * NY * (NXh + 1);
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const long long row = (long long)(j + r * T) * (NXh + 1);
        if (dcn) {
            float2 g0 = cscale(acc[r], scale), gn = cscale(accN[r], scale);
            if (accumulate) {
                g0 = cadd(g0, dk[row]);
                gn = cadd(gn, dk[row + NXh]);
            }
            dk[row] = g0;
            dk[row + NXh] = gn;
        } else if (cv) {
            float2 g = cscale(acc[r], 2.f * scale);
            if (accumulate) g = cadd(g, dk[row + col]);
            dk[row + col] = g;
        }
    }
}

// dw: grid (ceil(npairs / FPC), m).  Qf: [nb][m][nrows][NXh] packed row spectra
// of conj(hhat_k) . R_b (every row).  dw: [m][nrows][NX]; accumulate adds.
template <int NX>
__global__ void __launch_bounds__(256)
k_rows_grad_w(const float2* __restrict__ Qf, long long q_bstride, long long q_kstride, int nrows,
              int nb, const float* __restrict__ u, long long u_bstride, float* __restrict__ dw,
              float scale, int accumulate, const float2* __restrict__ tw) {
    constexpr int T = NX / kR;
    constexpr int FPC = 256 / T;
    constexpr int NXh = NX / 2;
    __shared__ float2 sbuf[FPC * fft_region(NX)];
    const int slot = threadIdx.x / T;
    const int j = threadIdx.x - slot * T;
    float2* b0 = sbuf + slot * fft_region(NX);
    float2* b1 = b0 + pad_len(NX);
    const int p = blockIdx.x * FPC + slot;
    const int k = blockIdx.y;
    const int ga = 2 * p, gb = ga + 1;
    const bool va = ga < nrows, vb = gb < nrows;

    auto load = [&](int b, float2 (&v)[kR], float (&ua)[kR], float (&ub)[kR]) {
        const float2* pa = Qf + b * q_bstride + k * q_kstride + (long long)(va ? ga : 0) * NXh;
        const float2* pb = Qf + b * q_bstride + k * q_kstride + (long long)(vb ? gb : 0) * NXh;
        const float* sa = u + b * u_bstride + (long long)(va ? ga : 0) * NX;
        const float* sb = u + b * u_bstride + (long long)(vb ? gb : 0) * NX;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int f = j + r * T;
            const float2 xa = va ? load_half<NX>(pa, f) : make_float2(0.f, 0.f);
            const float2 xb = vb ? load_half<NX>(pb, f) : make_float2(0.f, 0.f);
            v[r] = make_float2(xa.x - xb.y, xa.y + xb.x);
            ua[r] = va ? __ldg(sa + f) : 0.f;
            ub[r] = vb ? __ldg(sb + f) : 0.f;
        }
    };
    float2 acc[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) acc[r] = make_float2(0.f, 0.f);
    float2 v[kR];
    float ua[kR], ub[kR];
    load(0, v, ua, ub);
    for (int b = 0; b < nb; ++b) {
        const bool more = b + 1 < nb;
        float2 vn[kR];
        float uan[kR], ubn[kR];
        if (more) load(b + 1, vn, uan, ubn);
        fft<NX, true>(v, j, b0, b1, tw);
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            acc[r].x = fmaf(ua[r], v[r].x, acc[r].x);
            acc[r].y = fmaf(ub[r], v[r].y, acc[r].y);
        }
        if (more) {
#pragma unroll
            for (int r = 0; r < kR; ++r) {
                v[r] = vn[r];
                ua[r] = uan[r];
                ub[r] = ubn[r];
            }
        }
    }
    float* da = dw + ((long long)k * nrows + ga) * NX;
    float* db = dw + ((long long)k * nrows + gb) * NX;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int n = j + r * T;
        if (va) da[n] = acc[r].x * scale + (accumulate ? da[n] : 0.f);
        if (vb) db[n] = acc[r].y * scale + (accumulate ? db[n] : 0.f);
    }
}

// ------------------------------------------------------------------- 1D
template <int N, int WIDE = 0>
struct Cfg1d {
    static constexpr int T = N / kR;
    // FFT slots per CTA: 256 threads (throughput), or with WIDE up to 8 slots
    // in up to 1024 threads, so that a few right-hand sides finish sooner (the
    // slots work on different term pairs of the same right-hand side)
    static constexpr int G = WIDE ? ((1024 / T) < 8 ? ((1024 / T) > 0 ? 1024 / T : 1) : 8)
                                  : ((256 / T) > 0 ? (256 / T) : 1);
    static constexpr int NT = T * G;
    static constexpr int SMEM = G * fft_region(N) * (int)sizeof(float2);
};

// Ask L2 for the `bytes` at p (one 128-byte line per thread of the CTA), so that
// a latency-bound CTA finds them there when it reaches their loads.
__device__ __forceinline__ void prefetch_l2_block(const void* p, long long bytes) {
    const char* c = static_cast<const char*>(p);
    for (long long o = 128ll * threadIdx.x; o < bytes; o += 128ll * blockDim.x)
        asm volatile("prefetch.global.L2 [%0];\n" ::"l"(c + o));
}

// y_b = (1/N) C2R( sum_k hhat_k . R2C(w_k . u_b) ).  One CTA per b; each
// slot takes pairs of terms (w_k u + i w_{k+1} u in one complex FFT) and
// accumulates the half spectrum in registers; the slots' sums are reduced in
// shared memory and one inverse FFT follows.  hp: [m][N/2] packed spectra.
template <int N, typename WT = float, typename HT = float2, int WIDE = 0>
__global__ void __launch_bounds__(Cfg1d<N, WIDE>::NT)
k_fwd_1d(const float* __restrict__ u, const WT* __restrict__ w,
         const HT* __restrict__ hp, const float* __restrict__ hscale, int m, float* __restrict__ y, float scale,
         const float2* __restrict__ tw) {
    using CF = Cfg1d<N, WIDE>;
    constexpr int T = CF::T;
    constexpr int G = CF::G;
    constexpr int Nh = N / 2;
    extern __shared__ float2 smem[];
    const int slot = threadIdx.x / T;
    const int j = threadIdx.x - slot * T;
    float2* b0 = smem + slot * fft_region(N);
    float2* b1 = b0 + pad_len(N);
    const int b = blockIdx.x;
    // the twiddles and spectra are read stage by stage and after the first FFT:
    // with few right-hand sides (a latency-bound launch) start them towards L2 now
    if (gridDim.x <= 8) {
        prefetch_l2_block(tw, (long long)FftPlan<N>::TWLEN * sizeof(float2));
        prefetch_l2_block(hp, (long long)m * Nh * sizeof(HT));
    }
    const float* ub = u + (long long)b * N;
    float ureg[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) ureg[r] = __ldg(ub + j + r * T);
    float2 acc[kR / 2];
#pragma unroll
    for (int r = 0; r < kR / 2; ++r) acc[r] = make_float2(0.f, 0.f);

    const int npairs = (m + 1) / 2;
    const int iters = (npairs + G - 1) / G;
    for (int it = 0; it < iters; ++it) {
        const int pr = it * G + slot;
        const bool a0 = pr < npairs;
        const int k0 = 2 * pr, k1 = k0 + 1;
        const bool a1 = a0 && k1 < m;
        float2 v[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int n = j + r * T;
            v[r] = make_float2(a0 ? ldw(w + (long long)k0 * N + n) * ureg[r] : 0.f,
                               a1 ? ldw(w + (long long)k1 * N + n) * ureg[r] : 0.f);
        }
        fft<N, false>(v, j, b0, b1, tw);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kR; ++r) b0[padi(j + r * T)] = v[r];
        __syncthreads();
        if (a0) {
            const HT* h0 = hp + (long long)k0 * Nh;
            const HT* h1 = hp + (long long)(a1 ? k1 : k0) * Nh;
            const float s0 = hscale_of<HT>(hscale, k0);
            const float s1 = hscale_of<HT>(hscale, a1 ? k1 : k0);
#pragma unroll
            for (int r = 0; r < kR / 2; ++r) {
                const int f = j + r * T;
                if (f == 0) {
                    // the DC and Nyquist terms are real: acc[0] of thread 0 packs (DC, Nyquist)
                    const float2 p0 = ldh(&h0[0], s0);
                    acc[0].x = fmaf(p0.x, v[0].x, acc[0].x);
                    acc[0].y = fmaf(p0.y, v[kR / 2].x, acc[0].y);
                    if (a1) {
                        const float2 p1 = ldh(&h1[0], s1);
                        acc[0].x = fmaf(p1.x, v[0].y, acc[0].x);
                        acc[0].y = fmaf(p1.y, v[kR / 2].y, acc[0].y);
                    }
                } else {
                    float2 A, B;
                    split_dc_nyq(v[r], b0[padi(N - f)], A, B);
                    acc[r] = cfma(ldh(&h0[f], s0), A, acc[r]);
                    if (a1) acc[r] = cfma(ldh(&h1[f], s1), B, acc[r]);
                }
            }
        }
    }
    // reduce over slots into slot 0's second buffer (packed half spectrum)
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kR / 2; ++r) b0[j + r * T] = acc[r];
    __syncthreads();
    float2* red = smem + pad_len(N);
    if (slot == 0) {
#pragma unroll
        for (int r = 0; r < kR / 2; ++r) {
            float2 s = smem[j + r * T];
            for (int g = 1; g < G; ++g) s = cadd(s, smem[g * fft_region(N) + j + r * T]);
            red[j + r * T] = s;
        }
    }
    __syncthreads();
    float2 v[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r)
        v[r] = (slot == 0) ? load_half<N>(red, j + r * T) : make_float2(0.f, 0.f);
    fft<N, true>(v, j, b0, b1, tw);
    if (slot == 0) {
        float* yb = y + (long long)b * N;
#pragma unroll
        for (int r = 0; r < kR; ++r) yb[j + r * T] = v[r].x * scale;
    }
}

// x_b = (1/N) sum_k w_k . IFFT( conj(hhat_k) . FFT(v_b) ).  One CTA per b;
// every slot forms FFT(v_b) and takes pairs of terms: the two inverse FFTs
// of a pair are real, so they share one complex inverse FFT.
template <int N, typename WT = float, typename HT = float2, int WIDE = 0>
__global__ void __launch_bounds__(Cfg1d<N, WIDE>::NT)
k_adj_1d(const float* __restrict__ vin, const WT* __restrict__ w,
         const HT* __restrict__ hp, const float* __restrict__ hscale, int m, float* __restrict__ x, float scale,
         const float2* __restrict__ tw) {
    using CF = Cfg1d<N, WIDE>;
    constexpr int T = CF::T;
    constexpr int G = CF::G;
    constexpr int Nh = N / 2;
    extern __shared__ float2 smem[];
    const int slot = threadIdx.x / T;
    const int j = threadIdx.x - slot * T;
    float2* b0 = smem + slot * fft_region(N);
    float2* b1 = b0 + pad_len(N);
    const int b = blockIdx.x;
    // the twiddles, spectra and windows are read stage by stage and after the
    // FFT of v: with few right-hand sides (a latency-bound launch) start them
    // towards L2 now
    if (gridDim.x <= 8) {
        prefetch_l2_block(tw, (long long)FftPlan<N>::TWLEN * sizeof(float2));
        prefetch_l2_block(hp, (long long)m * Nh * sizeof(HT));
        prefetch_l2_block(w, (long long)m * N * sizeof(WT));
    }
    const float* vb = vin + (long long)b * N;
    float2 V[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) V[r] = make_float2(__ldg(vb + j + r * T), 0.f);
    fft<N, false>(V, j, b0, b1, tw);
    float ax[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) ax[r] = 0.f;

    const int npairs = (m + 1) / 2;
    const int iters = (npairs + G - 1) / G;
    for (int it = 0; it < iters; ++it) {
        const int pr = it * G + slot;
        const bool a0 = pr < npairs;
        const int k0 = 2 * pr, k1 = k0 + 1;
        const bool a1 = a0 && k1 < m;
        const HT* h0 = hp + (long long)(a0 ? k0 : 0) * Nh;
        const HT* h1 = hp + (long long)(a1 ? k1 : 0) * Nh;
        const float s0 = hscale_of<HT>(hscale, a0 ? k0 : 0);
        const float s1 = hscale_of<HT>(hscale, a1 ? k1 : 0);
        float2 p[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int f = j + r * T;
            float2 t = make_float2(0.f, 0.f);
            if (a0) t = cmulc(V[r], load_half_h<N, HT>(h0, f, s0));
            if (a1) {
                const float2 s = cmulc(V[r], load_half_h<N, HT>(h1, f, s1));
                t.x -= s.y;
                t.y += s.x;
            }
            p[r] = t;
        }
        fft<N, true>(p, j, b0, b1, tw);
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int n = j + r * T;
            if (a0) ax[r] = fmaf(ldw(w + (long long)k0 * N + n), p[r].x, ax[r]);
            if (a1) ax[r] = fmaf(ldw(w + (long long)k1 * N + n), p[r].y, ax[r]);
        }
    }
    __syncthreads();
    float* fb = reinterpret_cast<float*>(b0);
#pragma unroll
    for (int r = 0; r < kR; ++r) fb[j + r * T] = ax[r];
    __syncthreads();
    if (slot == 0) {
        float* xb = x + (long long)b * N;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            float s = fb[j + r * T];
            for (int g = 1; g < G; ++g)
                s += reinterpret_cast<const float*>(smem + g * fft_region(N))[j + r * T];
            xb[j + r * T] = s * scale;
        }
    }
}

// Plan (1D): packed R2C spectra of the impulse responses, two per complex
// FFT (h_k + i h_{k+1}).  Grid: ceil(ceil(m/2) / G).
template <int N>
__global__ void __launch_bounds__(Cfg1d<N>::NT)
k_spec_1d(const float* __restrict__ h, int m, float2* __restrict__ hp,
          const float2* __restrict__ tw) {
    using CF = Cfg1d<N>;
    constexpr int T = CF::T;
    constexpr int G = CF::G;
    constexpr int Nh = N / 2;
    extern __shared__ float2 smem[];
    const int slot = threadIdx.x / T;
    const int j = threadIdx.x - slot * T;
    float2* b0 = smem + slot * fft_region(N);
    float2* b1 = b0 + pad_len(N);
    const int pr = blockIdx.x * G + slot;
    const int k0 = 2 * pr, k1 = k0 + 1;
    const bool a0 = k0 < m, a1 = k1 < m;
    float2 v[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int n = j + r * T;
        v[r] = make_float2(a0 ? __ldg(h + (long long)k0 * N + n) : 0.f,
                           a1 ? __ldg(h + (long long)k1 * N + n) : 0.f);
    }
    fft<N, false>(v, j, b0, b1, tw);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kR; ++r) b0[padi(j + r * T)] = v[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kR / 2; ++r) {
        const int f = j + r * T;
        float2 A, B;
        if (f == 0) {
            A = make_float2(v[0].x, v[kR / 2].x);
            B = make_float2(v[0].y, v[kR / 2].y);
        } else {
            split_dc_nyq(v[r], b0[padi(N - f)], A, B);
        }
        if (a0) hp[(long long)k0 * Nh + f] = A;
        if (a1) hp[(long long)k1 * Nh + f] = B;
    }
}

// 1D backward for term k = blockIdx.x: dhhat_k (natural [N/2+1]) and dw_k
// ([N]); slots take right-hand sides.  w_k . u_b + i r_b share one FFT; the
// inverse FFT of conj(hhat_k) . R_b gives the correlation of r_b with h_k.
template <int N>
__global__ void __launch_bounds__(Cfg1d<N>::NT)
k_grad_1d(const float* __restrict__ u, const float* __restrict__ rr, const float* __restrict__ w,
          const float2* __restrict__ hp, int nb, float2* __restrict__ dh, float* __restrict__ dw,
          float scale, int accumulate, const float2* __restrict__ tw) {
    using CF = Cfg1d<N>;
    constexpr int T = CF::T;
    constexpr int G = CF::G;
    constexpr int Nh = N / 2;
    extern __shared__ float2 smem[];
    const int slot = threadIdx.x / T;
    const int j = threadIdx.x - slot * T;
    float2* b0 = smem + slot * fft_region(N);
    float2* b1 = b0 + pad_len(N);
    const int k = blockIdx.x;
    const float2* hk = hp + (long long)k * Nh;
    float wk[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) wk[r] = __ldg(w + (long long)k * N + j + r * T);
    float2 ah[kR / 2];
    float aw[kR];
    float ahn = 0.f;   // Nyquist (thread j = 0)
#pragma unroll
    for (int r = 0; r < kR / 2; ++r) ah[r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < kR; ++r) aw[r] = 0.f;
    const int iters = (nb + G - 1) / G;
    for (int it = 0; it < iters; ++it) {
        const int b = it * G + slot;
        const bool act = b < nb;
        float2 v[kR];
        float ub[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int n = j + r * T;
            ub[r] = act ? __ldg(u + (long long)b * N + n) : 0.f;
            v[r] = make_float2(wk[r] * ub[r], act ? __ldg(rr + (long long)b * N + n) : 0.f);
        }
        fft<N, false>(v, j, b0, b1, tw);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kR; ++r) b0[padi(j + r * T)] = v[r];
        __syncthreads();
        float2 p[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int f = j + r * T;
            float2 X, R;
            split_dc_nyq(v[r], b0[padi((N - f) & (N - 1))], X, R);
            if (r < kR / 2) {
                if (f == 0) {
                    ah[0].x = fmaf(R.x, X.x, ah[0].x);
                } else {
                    ah[r] = cfmac(X, R, ah[r]);
                }
            }
            if (f == Nh) ahn = fmaf(R.x, X.x, ahn);
            p[r] = cmulc(R, load_half<N>(hk, f));
        }
        fft<N, true>(p, j, b0, b1, tw);
#pragma unroll
        for (int r = 0; r < kR; ++r) aw[r] = fmaf(ub[r], p[r].x, aw[r]);
    }
    // reduce over slots: half spectrum into b0 (float2), window gradient into b1 (float)
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kR / 2; ++r) b0[j + r * T] = ah[r];
    if (j == 0) b0[Nh] = make_float2(ahn, 0.f);
    float* fw = reinterpret_cast<float*>(b1);
#pragma unroll
    for (int r = 0; r < kR; ++r) fw[j + r * T] = aw[r];
    __syncthreads();
    if (slot == 0) {
        float2* dk = dh + (long long)k * (Nh + 1);
        float* wk_out = dw + (long long)k * N;
#pragma unroll
        for (int r = 0; r < kR / 2; ++r) {
            const int f = j + r * T;
            float2 s = smem[f];
            for (int g = 1; g < G; ++g) s = cadd(s, smem[g * fft_region(N) + f]);
            float2 out = f == 0 ? make_float2(s.x * scale, 0.f) : cscale(s, 2.f * scale);
            if (accumulate) out = cadd(out, dk[f]);
            dk[f] = out;
        }
        if (j == 0) {
            float sn = smem[Nh].x;
            for (int g = 1; g < G; ++g) sn += smem[g * fft_region(N) + Nh].x;
            float2 out = make_float2(sn * scale, 0.f);
            if (accumulate) out = cadd(out, dk[Nh]);
            dk[Nh] = out;
        }
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int n = j + r * T;
            float s = fw[n];
            for (int g = 1; g < G; ++g)
                s += reinterpret_cast<const float*>(smem + g * fft_region(N) + pad_len(N))[n];
            wk_out[n] = s * scale + (accumulate ? wk_out[n] : 0.f);
        }
    }
}

}  // namespace pce
