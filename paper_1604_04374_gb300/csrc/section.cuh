// section.cuh -- sectioned apply (Lemma 3.2): every term is convolved on
// sections of LR x LC points (LR = 1024 rows, LC a power of two chosen at plan
// time), each holding a column tile of the window box of w_k plus the support
// of h_k, and the results are added into the output (overlap-add), instead of
// transforming the whole grid once per term.  Sections are indexed by s; the
// geometry of section s (SecGeom) names its term k.
//
// Coordinates.  A section's tile of the box starts at grid (r0, c0) (its
// columns [c0, c0 + nc) are box columns of the term; tiles of one term take
// consecutive column ranges); section offsets rho are relative to it.  h_k's support, as signed offsets, is [dr0, dr0 + snr) x
// [dc0, dc0 + snc).  h_k is placed at section position (d mod LR, d mod LC);
// a section position holds box offset rho at rho mod LR (LC).
//   forward:  input rows rho in [0, nr),   columns [0, nc)   (times w_k)
//             output rows [dr0, nr - 1 + dr0 + snr - 1], columns likewise
//   adjoint:  input = the forward output window, output = the box (times w_k)
// Every window is at most LR (LC) long, so no section position is used twice:
// the circular convolution of the section is the linear one.
//
// Kernels (one warp per 1024-point column, Stockham FFTs for the rows):
//   k_sec_r2c:  rows of the input window gathered from the grid (w_k applied
//               in the forward), R2C, packed half spectra [b][s][row][LC/2]
//   kw_sec_cols: per section and column, FFT_y, times the section spectrum of
//               h_k (conjugated for the adjoint; copied into shared memory
//               by the TMA engine once per CTA), IFFT_y, output rows
//   k_sec_c2r:  C2R of the output rows, times 1 / (LR LC) (and w_k in the
//               adjoint), added into the grid with atomicAdd (terms overlap)
#pragma once

#include "kernels.cuh"
#include "wkernels.cuh"

namespace pce {

constexpr int kSecLR = 1024;

// box offset held at section position n of a window [lo, hi] (hi - lo < L), or
// a value outside the window
__device__ __forceinline__ int sec_offset(int n, int lo, int hi, int L) { return n <= hi ? n : n - L; }

// Grid column of section column offset rc: c0 is in [0, n) and |rc| < L, so
// for sections no wider than the grid (L <= n) one conditional add or
// subtract wraps it; wider sections (small grids) take the remainder.
__device__ __forceinline__ int sec_col(int c0, int rc, int n, bool narrow) {
    int c = c0 + rc;
    if (narrow) {
        c += c < 0 ? n : 0;
        c -= c >= n ? n : 0;
        return c;
    }
    return (c % n + n) % n;
}

// Input rows: items (k, q) take window rows 2q, 2q+1 of term k.
template <int NX, bool WIN, typename WT = float>
__global__ void __launch_bounds__(256)
k_sec_r2c(const float* __restrict__ src, long long src_bstride, int NYg, int NXg,
          const WT* __restrict__ wbox, const SecGeom* __restrict__ geo, const int2* __restrict__ items,
          int nitems, float2* __restrict__ dst, long long dst_bstride, long long dst_kstride,
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
    const int item = blockIdx.x * FPC + slot;
    const bool active = item < nitems;
    const int2 kq = active ? items[item] : make_int2(0, 0);
    const SecGeom g = geo[kq.x];
    const bool narrow = NX <= NXg;
    const int ia = 2 * kq.y, ib = ia + 1;
    const bool va = active && ia < g.in_rows, vb = active && ib < g.in_rows;
    const int ra = g.in_lo_r + ia, rb = g.in_lo_r + ib;   // box row offsets
    const float* srcb = src + b * src_bstride;
    const float* sa = srcb + (long long)(((g.r0 + ra) % NYg + NYg) % NYg) * NXg;
    const float* sb = srcb + (long long)(((g.r0 + rb) % NYg + NYg) % NYg) * NXg;
    float2 v[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int n = j + r * T;
        const int rc = sec_offset(n, g.in_lo_c, g.in_hi_c, NX);
        float xa = 0.f, xb = 0.f;
        if (rc >= g.in_lo_c && rc <= g.in_hi_c) {
            const int col = sec_col(g.c0, rc, NXg, narrow);
            if (va) xa = __ldg(sa + col);
            if (vb) xb = __ldg(sb + col);
            if (WIN) {
                if (va) xa *= ldw(wbox + g.woff + (long long)ra * g.ldw + rc);
                if (vb) xb *= ldw(wbox + g.woff + (long long)rb * g.ldw + rc);
            }
        }
        v[r] = make_float2(xa, xb);
    }
    fft<NX, false>(v, j, b0, b1, tw);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kR; ++r) b0[padi(j + r * T)] = v[r];
    __syncthreads();
    float2* da = dst + b * dst_bstride + kq.x * dst_kstride + (long long)ia * NXh;
    float2* db = dst + b * dst_bstride + kq.x * dst_kstride + (long long)ib * NXh;
#pragma unroll
    for (int r = 0; r < kR / 2; ++r) {
        const int f = j + r * T;
        float2 A, B;
        if (f == 0) {
            A = make_float2(v[0].x, v[kR / 2].x);
            B = make_float2(v[0].y, v[kR / 2].y);
        } else {
            split_dc_nyq(v[r], b0[padi(NX - f)], A, B);
        }
        if (va) da[f] = A;
        if (vb) db[f] = B;
    }
}

// Columns of the sections (LR = 1024).  Grid (sections, ceil(NXh / 4)), 128
// threads, kSecColSmem bytes; each CTA takes one section and four columns and
// runs all nb right-hand sides through them.  hsT: the section spectra of h_k,
// [m][NXh][1024] (c = 0: DC column), hsN: [m][1024] (Nyquist); float2, or
// half2 times hscale[k] (reduced storage).  A warp's spectrum column (8 KB)
// is copied once per CTA into a buffer of its own by the TMA engine, at the
// start, and serves every right-hand side (several sections of a term read
// the same columns, so per-right-hand-side copies multiplied the traffic);
// the one wait for it is bounded (status bit kStatusTimeout, products skipped
// after it).  Shared memory: the staging tile, whose four quarters double as
// the warps' transpose tiles, and the spectrum buffers (64 KB, three CTAs per
// SM at up to 168 registers).
constexpr int kSecColSmem = kSecLR * kWColWarps * 8 + kWColWarps * kSecLR * 8;
template <bool CONJ, typename HT = float2>
__global__ void __launch_bounds__(kWColWarps * 32, 3)
kw_sec_cols(const float2* __restrict__ Z, long long z_bstride, long long z_kstride, int nb,
            const HT* __restrict__ hsT, const HT* __restrict__ hsN, const float* __restrict__ hscale,
            const SecGeom* __restrict__ geo,
            int NXh, float2* __restrict__ A, long long a_bstride, long long a_kstride,
            const float2* __restrict__ tw, int* __restrict__ status, long long wait_limit, int skip_copy) {
    constexpr int NY = kSecLR;
    extern __shared__ float2 smem[];
    float2* tile = smem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* tr = smem + warp * kWarpN;   // a quarter of the staging tile
    const int sec = blockIdx.x;   // section; its term is g.k
    const int col0 = blockIdx.y * kWColWarps;
    const int col = col0 + warp;
    const bool cv = col < NXh;
    const bool dcn = blockIdx.y == 0 && warp == 0;
    const SecGeom g = geo[sec];
    const int k = g.k;
    __shared__ unsigned long long bars[kWColWarps];
    unsigned long long* bar = &bars[warp];
    if (lane == 0) mbar_init(bar);
    __syncwarp();
    unsigned parity = 0;
    bool failed = false;
    const HT* hcol = hsT + ((long long)k * NXh + (cv ? col : 0)) * NY;
    const HT* h0 = hsT + (long long)k * NXh * NY;   // DC column (dcn warp only)
    const HT* hn = hsN + (long long)k * NY;
    const float sk = hscale_of<HT>(hscale, k);
    const int swl = tix_sw(lane, warp);
    HT* hb = reinterpret_cast<HT*>(smem + NY * kWColWarps) + warp * NY;
    const bool bulk = !dcn && cv;
    if (bulk && lane == 0) bulk_load(hb, hcol, NY * sizeof(HT), bar, skip_copy);
    for (int b = 0; b < nb; ++b) {
        // the twiddles and the row indices are the same for every right-hand
        // side; opaque copies keep the compiler from holding them in registers
        // across the loop (which spills)
        const float2* twb = tw;
        int lo_r = g.in_lo_r, rows = g.in_rows;
        asm volatile("" : "+l"(twb), "+r"(lo_r), "+r"(rows));
        tile_load(tile, Z + b * z_bstride + sec * z_kstride, g.in_rows, NXh, col0);
        cp_async_wait_all();
        __syncthreads();
        float2 v[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int i = wrap(lane + 32 * q - lo_r, NY);
            v[q] = (i < rows) ? tile[tix(i, warp)] : make_float2(0.f, 0.f);
        }
        __syncthreads();   // every warp has read its rows: the transpose tiles are free
        warp_fft1024<false>(v, tr, twb);
        if (bulk && b == 0) {
            if (!mbar_wait(bar, parity, wait_limit)) {
                failed = true;
                if (lane == 0) atomicOr(status, kStatusTimeout);
                // the copy may still be in flight into the buffer: wait once more
                // (bounded) before the kernel goes on; the products are skipped
                mbar_wait(bar, parity, wait_limit);
            }
            parity ^= 1;
        }
        if (dcn) {
            // the partner values Z[-f] come from the transpose tile (free after the
            // FFT), so the products can overwrite v in place
#pragma unroll
            for (int mm = 0; mm < 32; ++mm) tr[lane + 32 * mm] = v[mm];
            __syncwarp();
#pragma unroll
            for (int mm = 0; mm < 32; ++mm) {
                const int f = lane + 32 * mm;
                float2 a, bb;
                split_dc_nyq(v[mm], tr[(NY - f) & (NY - 1)], a, bb);
                const float2 hd = CONJ ? cconj(ldh(&h0[f], sk)) : ldh(&h0[f], sk);
                const float2 hN = CONJ ? cconj(ldh(&hn[f], sk)) : ldh(&hn[f], sk);
                float2 t = cmul(hd, a);
                const float2 sN = cmul(hN, bb);
                t.x -= sN.y;
                t.y += sN.x;
                v[mm] = t;
            }
            __syncwarp();
        } else if (cv && !failed) {
#pragma unroll
            for (int mm = 0; mm < 32; ++mm) {
                const float2 hv = lds_h(&hb[lane + 32 * mm], sk);
                v[mm] = CONJ ? cmulc(v[mm], hv) : cmul(v[mm], hv);
            }
        } else {
#pragma unroll
            for (int mm = 0; mm < 32; ++mm) v[mm] = make_float2(0.f, 0.f);
        }
        warp_fft1024<true>(v, tr, twb);
        __syncthreads();   // every warp is done with its transpose tile
#pragma unroll
        for (int q = 0; q < 32; ++q) tile[4 * (lane + 32 * q) + swl] = v[q];
        __syncthreads();
        float2* Ab = A + b * a_bstride + sec * a_kstride;
        for (int e = threadIdx.x; e < g.out_rows * kWColWarps; e += kWColWarps * 32) {
            const int i = e >> 2, c = e & 3;
            const int s = wrap(g.out_lo_r + i, NY);
            if (col0 + c < NXh) Ab[(long long)i * NXh + col0 + c] = tile[tix(s, c)];
        }
        __syncthreads();   // the store has read the tile before the next right-hand side's load
    }
}

// Output rows: items (k, q) take output-window rows 2q, 2q+1 of term k; C2R,
// times scale (and the window in the adjoint), added into the grid.
template <int NX, bool WIN, typename WT = float>
__global__ void __launch_bounds__(256)
k_sec_c2r(const float2* __restrict__ src, long long src_bstride, long long src_kstride,
          const SecGeom* __restrict__ geo, const int2* __restrict__ items, int nitems,
          const WT* __restrict__ wbox, float* __restrict__ dst, long long dst_bstride, int NYg, int NXg,
          float scale, const float2* __restrict__ tw) {
    constexpr int T = NX / kR;
    constexpr int FPC = 256 / T;
    constexpr int NXh = NX / 2;
    __shared__ float2 sbuf[FPC * fft_region(NX)];
    const int slot = threadIdx.x / T;
    const int j = threadIdx.x - slot * T;
    float2* b0 = sbuf + slot * fft_region(NX);
    float2* b1 = b0 + pad_len(NX);
    const int b = blockIdx.y;
    const int item = blockIdx.x * FPC + slot;
    const bool active = item < nitems;
    const int2 kq = active ? items[item] : make_int2(0, 0);
    const SecGeom g = geo[kq.x];
    const bool narrow = NX <= NXg;
    const int ia = 2 * kq.y, ib = ia + 1;
    const bool va = active && ia < g.out_rows, vb = active && ib < g.out_rows;
    const float2* base = src + b * src_bstride + kq.x * src_kstride;
    const float2* pa = base + (long long)(va ? ia : 0) * NXh;
    const float2* pb = base + (long long)(vb ? ib : 0) * NXh;
    float2 v[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int f = j + r * T;
        const float2 xa = va ? load_half<NX>(pa, f) : make_float2(0.f, 0.f);
        const float2 xb = vb ? load_half<NX>(pb, f) : make_float2(0.f, 0.f);
        v[r] = make_float2(xa.x - xb.y, xa.y + xb.x);
    }
    const int ra = g.out_lo_r + ia, rb = g.out_lo_r + ib;   // box row offsets
    // window values (adjoint), loaded before the FFT so that their latency
    // overlaps it
    float wa[kR], wb[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        wa[r] = 1.f;
        wb[r] = 1.f;
        if (WIN) {
            const int rc = sec_offset(j + r * T, g.out_lo_c, g.out_hi_c, NX);
            const bool in = rc >= g.out_lo_c && rc <= g.out_hi_c;
            wa[r] = (in && va) ? ldw(wbox + g.woff + (long long)ra * g.ldw + rc) : 0.f;
            wb[r] = (in && vb) ? ldw(wbox + g.woff + (long long)rb * g.ldw + rc) : 0.f;
        }
    }
    fft<NX, true>(v, j, b0, b1, tw);
    float* db = dst + b * dst_bstride;
    float* ya = db + (long long)(((g.r0 + ra) % NYg + NYg) % NYg) * NXg;
    float* yb = db + (long long)(((g.r0 + rb) % NYg + NYg) % NYg) * NXg;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int n = j + r * T;
        const int rc = sec_offset(n, g.out_lo_c, g.out_hi_c, NX);
        if (rc < g.out_lo_c || rc > g.out_hi_c) continue;
        const int col = sec_col(g.c0, rc, NXg, narrow);
        const float xa = v[r].x * scale * wa[r], xb = v[r].y * scale * wb[r];
        if (va) atomicAdd(ya + col, xa);
        if (vb) atomicAdd(yb + col, xb);
    }
}

}  // namespace pce
