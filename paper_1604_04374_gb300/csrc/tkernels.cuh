// tkernels.cuh -- column kernels of separable plans for Ny = 1024 with the
// per-warp state in tensor memory.
//
// They compute exactly what kw_cols_fwd<float2, true> / kw_cols_adj<false,
// float2, true> (wkernels.cuh) compute, with the same global layouts, and run
// the same one-warp 1024-point FFT (warpfft.cuh).  What moves is the state a
// warp carries from term to term:
//
//   forward: the slot's column Z_j[:, c] (reused by every term of the slot)
//            and the spectral accumulator sum_k hhat_k . FFT_y(wy_k . Z_j);
//   adjoint: the column spectrum FFT_y(V[:, c]) (reused by every term) and
//            the slot accumulator S_j = sum_k wy_k . IFFT_y(conj(hhat_k) V).
//
// In wkernels.cuh the accumulator takes 64 registers per thread beside the
// 64 of the FFT, and the column lives in a 32 KB shared tile per CTA: 168
// registers and 72 KB per 4-warp CTA, so 3 CTAs (12 warps) per SM.  Here both
// live in tensor memory, 64 + 64 columns of the warp's lane quarter
// (tmem.cuh), and the shared memory holds only the four warps' transpose tiles
// (which double as the staging tile of the coalesced column loads and stores)
// and the row factors: 40 KB and 4 CTAs (16 warps) per SM, bounded by the
// 512 tensor-memory columns of an SM (4 x 128).  The shared-memory request is
// padded so that a fifth CTA never fits: every resident CTA's allocation is
// then satisfied at once.
//
// Layout of a warp's 128 columns: [0, 64) held column, [64, 128) accumulator;
// thread l holds, like the registers of the one-warp FFT, the values of rows
// (or frequencies) l + 32 q at columns 2q, 2q + 1.
//
// PRUNE (every term's row factor wy_k nonzero only inside rows
// [s_k, s_k + 512) mod 1024, s_k = 32 q0_k; the hats of a 4 x 4 node grid
// cover 511 rows): the forward column input of a term is zero on half of the
// column, the adjoint needs the term's inverse FFT on half of the rows only
// (Lemma 3.2 applied to the column transforms).  With the input rotated by
// s_k, the nonzeros land in q < 16 of every lane, and the first 32-point DFT
// of the one-warp FFT skips its first butterflies (warpfft.cuh, IN_HALF); in
// the adjoint the last 32-point DFT computes outputs m < 16 only (OUT_HALF).
// The rotation costs nothing at apply time: FFT(x)[f] = W^{f s} FFT(x')[f]
// for x'[n] = x[n + s], so the plan stores hhat_k[f] W1024^{f s_k} (the
// forward then accumulates hhat'_k FFT(x'_k), and conj(hhat'_k) V shifts the
// adjoint's inverse FFT output by s_k).  The held column is read rotated from
// tensor memory at runtime column offsets (tm_load16_rot).
#pragma once

#include "tmem.cuh"
#include "wkernels.cuh"

namespace pce {

// tensor-memory columns of a CTA for columns of NY points: per warp NY / 16
// for the held column and as many for the accumulator (128 at 1024 points, 64
// at 512), over the warp's lane quarter
template <int NY>
__host__ __device__ constexpr int kt_tm_cols() { return 4 * (NY / 32); }
constexpr int kTmCols = kt_tm_cols<1024>();
// the four-step twiddles: 31 table loads per FFT (false) or ten loads and 21
// products (true, warpfft.cuh)
constexpr bool kTmSplit = false;
// four transpose tiles and two row-factor buffers
template <int NY>
__host__ __device__ constexpr int kt_smem_used() { return (kWColWarps * NY) * (int)sizeof(float2) + 2 * NY * (int)sizeof(float); }
// padded so that no more CTAs fit on an SM than its 512 tensor-memory columns
// serve (then every resident CTA's allocation is satisfied at once):
// 1024 points: 5 x (47 KB + the 1 KB per-CTA reserve) exceeds the SM's 228 KB,
// 4 x does not; 512 points: 9 x (25 + 1) KB exceeds it, 8 x does not
template <int NY>
__host__ __device__ constexpr int kt_smem() { return NY == 1024 ? 47 * 1024 : 25 * 1024; }
constexpr int kTColSmem = kt_smem<1024>();
static_assert(kt_smem<1024>() >= kt_smem_used<1024>() && kt_smem<512>() >= kt_smem_used<512>(),
              "tensor-memory column kernels: shared memory");
static_assert(512 / kt_tm_cols<1024>() == 4 && 512 / kt_tm_cols<512>() == 8,
              "tensor-memory column kernels: CTAs per SM by tensor memory");

// Allocate the CTA's tensor memory (warp 0), publish its base address and
// return this warp's lane-quarter base.
__device__ __forceinline__ unsigned tm_begin(unsigned* slot, int ncols) {
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tm_alloc(slot, ncols);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    return *slot + ((unsigned)(32 * warp) << 16);
}
// Every warp's tcgen05 loads and stores have completed (the loads wait in
// place; stores are waited by the caller).  Release the allocation (warp 0).
__device__ __forceinline__ void tm_end(const unsigned* slot, int ncols) {
    tm_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tm_fence_after();
        tm_dealloc(*slot, ncols);
    }
}

// A warp's column of QN complex values per lane (32 at 1024 points, 16 at 512)
// from / to tensor memory at columns taddr .. taddr + 2 QN
template <int QN>
__device__ __forceinline__ void tm_loadq(unsigned taddr, float2 (&v)[QN]) {
    if constexpr (QN == 32) {
        tm_load32c(taddr, v);
    } else {
#pragma unroll
        for (int h = 0; h < QN / 8; ++h) {
            float2 a[8];
            tm_load8c(taddr + 16 * h, a);
#pragma unroll
            for (int j = 0; j < 8; ++j) v[8 * h + j] = a[j];
        }
    }
}
template <int QN>
__device__ __forceinline__ void tm_storeq(unsigned taddr, const float2 (&v)[QN]) {
    if constexpr (QN == 32) {
        tm_store32c(taddr, v);
    } else {
#pragma unroll
        for (int h = 0; h < QN / 8; ++h) {
            float2 a[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = v[8 * h + j];
            tm_store8c(taddr + 16 * h, a);
        }
    }
}

// acc[8 quarter .. 8 quarter + 7] of a 32-value accumulator in tensor memory
template <typename F>
__device__ __forceinline__ void tm_update8(unsigned tacc, int quarter, F&& f) {
    float2 a[8];
    tm_load8c(tacc + 16 * quarter, a);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = f(8 * quarter + j, a[j]);
    tm_store8c(tacc + 16 * quarter, a);
}

// Rows i < nr of dst ([rows][NXh], columns col0 .. col0 + 3) from rows r0 + i
// (mod NY) of the CTA's swizzled staging tile.  Two columns per 16-byte store
// when dst is 16-byte aligned and NXh a multiple of 4 (always for power-of-two
// grids of 8 columns or more), else one per 8-byte store.
template <int NY = kWarpN>
__device__ __forceinline__ void store_cols(float2* __restrict__ dst, const float2* tile, int r0, int nr, int NXh,
                                           int col0) {
    if ((reinterpret_cast<unsigned long long>(dst) & 15) == 0 && (NXh & 3) == 0) {
        for (int e = threadIdx.x; e < nr * 2; e += kWColWarps * 32) {
            const int i = e >> 1, c = (e & 1) * 2;
            const int g = wrap(r0 + i, NY);
            const float2 x0 = tile[tix(g, c)], x1 = tile[tix(g, c + 1)];
            *reinterpret_cast<float4*>(dst + (long long)i * NXh + col0 + c) = make_float4(x0.x, x0.y, x1.x, x1.y);
        }
    } else {
        for (int e = threadIdx.x; e < nr * kWColWarps; e += kWColWarps * 32) {
            const int i = e >> 2, c = e & 3;
            if (col0 + c < NXh) dst[(long long)i * NXh + col0 + c] = tile[tix(wrap(r0 + i, NY), c)];
        }
    }
}

// X[(NY - f) mod NY] from a warp's transpose tile holding X[f] at f.
template <int NY = kWarpN>
__device__ __forceinline__ float2 tr_partner(const float2* tr, int f) { return tr[(NY - f) & (NY - 1)]; }

// F2 for separable plans, Ny = 1024.  Grid (batch, NXh / 4), 128 threads,
// kTColSmem bytes.  Arguments as kw_cols_fwd<float2, true>.
template <bool PRUNE, int NY = kWarpN>
__global__ void __launch_bounds__(kWColWarps * 32, NY == kWarpN ? 4 : 6)
kt_cols_fwd(const float2* __restrict__ Z, long long z_bstride, long long z_kstride,
            const float2* __restrict__ hhT, const float2* __restrict__ hN, const Box* __restrict__ box,
            int NXh, float2* __restrict__ A, long long a_bstride, const float2* __restrict__ tw,
            int* __restrict__ status, long long wait_limit, int skip_copy, SepTerms sep) {
    constexpr int QN = NY / 32;   // values per lane
    constexpr int NQ = QN / 8;    // quarters of eight
    extern __shared__ __align__(16) float2 smem[];
    float2* tile = smem;                                     // staging tile [1024][4] (swizzled)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* tr = smem + warp * NY;                       // this warp's transpose tile
    float* wys = reinterpret_cast<float*>(smem + NY * kWColWarps);
    __shared__ unsigned long long bars[kWColWarps];
    __shared__ unsigned tm_slot;
    const int b = blockIdx.x;
    const int col0 = blockIdx.y * kWColWarps;
    const int col = col0 + warp;
    const bool cv = col < NXh;
    const bool dcn = blockIdx.y == 0 && warp == 0;
    const float2* Zb = Z + b * z_bstride;
    unsigned long long* bar = &bars[warp];
    if (lane == 0) mbar_init(bar);
    const unsigned tbase = tm_begin(&tm_slot, kt_tm_cols<NY>());
    const unsigned t_hold = tbase, t_acc = tbase + 2 * QN;
    unsigned parity = 0;
    bool failed = false;
    const int swl = tix_sw(lane, warp);
    const int mode = sep.t1 < 0 ? kSepFinal : sep.mode;
    if (mode & kSepLoadAcc) {
        // slot-by-slot schedule: the frequency-domain sum of the earlier passes
        tile_load(tile, A + b * a_bstride, NY, NXh, col0);
        cp_async_wait_all();
        __syncthreads();
        float2 a[QN];
#pragma unroll
        for (int q = 0; q < QN; ++q) a[q] = tile[4 * (lane + 32 * q) + swl];
        tm_storeq<QN>(t_acc, a);
        tm_wait_st();
        __syncthreads();   // the staging tile is read: the transpose tiles are free again
    } else {
        float2 z[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) z[j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq) tm_store8c(t_acc + 16 * qq, z);
        tm_wait_st();
    }
    const int tbeg = sep.t1 < 0 ? 0 : sep.t0;
    const int tend = sep.t1 < 0 ? sep.nterms : sep.t1;
    if (tbeg < tend) {
        wy_load<NY>(wys + (tbeg & 1) * NY, sep.wrow, __ldg(&sep.korder[tbeg]));
        cp_async_commit();
    }
    int cur_slot = -1;
    for (int t = tbeg; t < tend; ++t) {
        const int k = __ldg(&sep.korder[t]);
        const int sl = __ldg(&sep.kslot[k]);
        cp_async_wait_all();
        __syncthreads();   // this term's row factors have landed; every warp is past its previous FFT
        if (sl != cur_slot) {   // uniform over the CTA: stage the slot's four columns, keep this warp's
            const Box bx = box[sl];
            tile_load(tile, Zb + sl * z_kstride, bx.nr, NXh, col0);
            cp_async_wait_all();
            __syncthreads();
            float2 v[QN];
            if (bx.r0 == 0 && bx.nr == NY) {
                const float2* tb = tile + 4 * lane + tix_sw(lane, warp);
#pragma unroll
                for (int q = 0; q < QN; ++q) v[q] = tb[128 * q];
            } else {
#pragma unroll
                for (int q = 0; q < QN; ++q) {
                    const int i = wrap(lane + 32 * q - bx.r0, NY);
                    v[q] = (i < bx.nr) ? tile[tix(i, warp)] : make_float2(0.f, 0.f);
                }
            }
            tm_storeq<QN>(t_hold, v);
            tm_wait_st();
            __syncthreads();   // the staging tile is read: the transpose tiles are free again
            cur_slot = sl;
        }
        // the next term's row factors into the other buffer (last read in the previous term)
        if (t + 1 < tend) {
            wy_load<NY>(wys + ((t + 1) & 1) * NY, sep.wrow, __ldg(&sep.korder[t + 1]));
            cp_async_commit();
        }
        float2 v[QN];
        {
            const float* wr = wys + (t & 1) * NY;
            if constexpr (PRUNE) {
                // rows 32 q0 + l + 32 j, j < 16: the support of wy_k, rotated to q < 16
                const int q0 = __ldg(&sep.kq0[k]);
                tm_load16_rot(t_hold, q0, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = cscale(v[j], wr[lane + 32 * ((q0 + j) & 31)]);
            } else {
                tm_loadq<QN>(t_hold, v);
#pragma unroll
                for (int q = 0; q < QN; ++q) v[q] = cscale(v[q], wr[lane + 32 * q]);
            }
        }
        const bool bulk = !dcn && cv && !failed;
        auto hook = [&] {
            if (bulk && lane == 0) bulk_load(tr, hhT + ((long long)k * NXh + col) * NY, NY * sizeof(float2), bar, skip_copy);
        };
        if constexpr (NY == kWarpN)
            warp_fft1024<false, kTmSplit, decltype(hook), PRUNE>(v, tr, tw, hook);
        else
            warp_fft512<false, kTmSplit, decltype(hook)>(v, tr, tw, hook);
        if (bulk) {
            if (!mbar_wait(bar, parity, wait_limit)) {
                failed = true;
                if (lane == 0) atomicOr(status, kStatusTimeout);
                // a copy may still be in flight into the tile: wait for it once
                // more (bounded) before the tile is reused; no further copies
                // are issued and the products are skipped from here on
                mbar_wait(bar, parity, wait_limit);
            }
            parity ^= 1;
        }
        if (dcn) {
            // the DC/Nyquist column: separate DC and Nyquist with the partner
            // frequencies, read back from the (unused) transpose tile
            const float2* h0 = hhT + (long long)k * NXh * NY;
            const float2* hn = hN + (long long)k * NY;
            __syncwarp();
#pragma unroll
            for (int mm = 0; mm < QN; ++mm) tr[lane + 32 * mm] = v[mm];
            __syncwarp();
#pragma unroll
            for (int qq = 0; qq < NQ; ++qq)
                tm_update8(t_acc, qq, [&](int mm, float2 a) {
                    const int f = lane + 32 * mm;
                    float2 x, y;
                    split_dc_nyq(v[mm], tr_partner<NY>(tr, f), x, y);
                    a = cfma(__ldg(&h0[f]), x, a);
                    const float2 s = cmul(__ldg(&hn[f]), y);
                    a.x -= s.y;
                    a.y += s.x;
                    return a;
                });
            tm_wait_st();
            __syncwarp();
        } else if (cv && !failed) {
#pragma unroll
            for (int qq = 0; qq < NQ; ++qq)
                tm_update8(t_acc, qq, [&](int mm, float2 a) { return cfma(tr[lane + 32 * mm], v[mm], a); });
            tm_wait_st();
        }
    }
    float2 acc[QN];
    tm_loadq<QN>(t_acc, acc);
    if (mode & kSepFinal) warp_fft<NY, true, kTmSplit>(acc, tr, tw);
    __syncthreads();   // every warp is done with its transpose tile: stage the four columns
#pragma unroll
    for (int mm = 0; mm < QN; ++mm) tile[4 * (lane + 32 * mm) + swl] = acc[mm];
    __syncthreads();
    store_cols<NY>(A + b * a_bstride, tile, 0, NY, NXh, col0);
    tm_end(&tm_slot, kt_tm_cols<NY>());
}

// G1b + G2 for separable plans, Ny = 1024.  Grid (batch, NXh / 4), 128
// threads, kTColSmem bytes.  Arguments as kw_cols_adj<false, float2, true>:
// Q receives, per slot, S_j on the slot box rows.
template <bool PRUNE, int NY = kWarpN>
__global__ void __launch_bounds__(kWColWarps * 32, NY == kWarpN ? 4 : 6)
kt_cols_adj(float2* __restrict__ V, long long v_bstride, const float2* __restrict__ hhT,
            const float2* __restrict__ hN, const Box* __restrict__ box, int NXh, float2* __restrict__ Q,
            long long q_bstride, long long q_kstride, const float2* __restrict__ tw, int* __restrict__ status,
            long long wait_limit, int skip_copy, SepTerms sep) {
    constexpr int QN = NY / 32;   // values per lane
    constexpr int NQ = QN / 8;    // quarters of eight
    extern __shared__ __align__(16) float2 smem[];
    float2* tile = smem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* tr = smem + warp * NY;
    float* wys = reinterpret_cast<float*>(smem + NY * kWColWarps);
    __shared__ unsigned long long bars[kWColWarps];
    __shared__ unsigned tm_slot;
    const int b = blockIdx.x;
    const int col0 = blockIdx.y * kWColWarps;
    const int col = col0 + warp;
    const bool cv = col < NXh;
    const bool dcn = blockIdx.y == 0 && warp == 0;
    const bool use_bulk = !dcn && cv;
    unsigned long long* bar = &bars[warp];
    if (lane == 0) mbar_init(bar);
    const unsigned tbase = tm_begin(&tm_slot, kt_tm_cols<NY>());
    const unsigned t_hold = tbase, t_acc = tbase + 2 * QN;
    unsigned parity = 0;
    bool failed = false;
    const int tbeg = sep.t1 < 0 ? 0 : sep.t0;
    const int tend = sep.t1 < 0 ? sep.nterms : sep.t1;
    const int mode = sep.t1 < 0 ? 0 : sep.mode;
    const int swl = tix_sw(lane, warp);

    if (tbeg < tend) wy_load<NY>(wys + (tbeg & 1) * NY, sep.wrow, __ldg(&sep.korder[tbeg]));
    tile_load(tile, V + b * v_bstride, NY, NXh, col0);
    cp_async_wait_all();
    __syncthreads();
    {
        float2 vv[QN];
#pragma unroll
        for (int q = 0; q < QN; ++q) vv[q] = tile[4 * (lane + 32 * q) + swl];
        __syncthreads();   // the staging tile is read: the transpose tiles are free
        const bool first_copy = use_bulk && tbeg < tend;
        if (mode & kSepSpecIn) {
            // an earlier pass stored the column spectrum: no FFT
            if (first_copy && lane == 0)
                bulk_load(tr, hhT + ((long long)__ldg(&sep.korder[tbeg]) * NXh + col) * NY, NY * sizeof(float2),
                          bar, skip_copy);
        } else {
            // the spectrum of the first term arrives while the FFT of V finishes
            // (after it, when the transpose tiles first stage the spectrum's store)
            auto hook0 = [&] {
                if (first_copy && !(mode & kSepSpecOut) && lane == 0)
                    bulk_load(tr, hhT + ((long long)__ldg(&sep.korder[tbeg]) * NXh + col) * NY, NY * sizeof(float2),
                              bar, skip_copy);
            };
            warp_fft<NY, false, kTmSplit, decltype(hook0)>(vv, tr, tw, hook0);
            if (mode & kSepSpecOut) {
                // the column spectrum back into V for the later passes (in place: this
                // CTA is the only reader of these four columns)
                __syncthreads();
#pragma unroll
                for (int q = 0; q < QN; ++q) tile[4 * (lane + 32 * q) + swl] = vv[q];
                __syncthreads();
                store_cols<NY>(V + b * v_bstride, tile, 0, NY, NXh, col0);
                __syncthreads();
                if (first_copy && lane == 0)
                    bulk_load(tr, hhT + ((long long)__ldg(&sep.korder[tbeg]) * NXh + col) * NY, NY * sizeof(float2),
                              bar, skip_copy);
            }
        }
        tm_storeq<QN>(t_hold, vv);
        tm_wait_st();
    }
    int prev_slot = -1;
    for (int t = tbeg; t < tend; ++t) {
        const int k = __ldg(&sep.korder[t]);
        const int sl = __ldg(&sep.kslot[k]);
        const int kn = t + 1 < tend ? __ldg(&sep.korder[t + 1]) : -1;   // within this pass
        const bool first = sl != prev_slot;
        const bool last = kn < 0 || __ldg(&sep.kslot[kn]) != sl;
        prev_slot = sl;
        if (use_bulk && !failed) {
            if (!mbar_wait(bar, parity, wait_limit)) {
                failed = true;
                if (lane == 0) atomicOr(status, kStatusTimeout);
                // a copy may still be in flight into the tile: wait for it once
                // more (bounded) before the tile is reused; no further copies
                // are issued and the products are skipped from here on
                mbar_wait(bar, parity, wait_limit);
            }
            parity ^= 1;
        }
        float2 p[QN];
        if (dcn) {
            tm_loadq<QN>(t_hold, p);
            const float2* h0 = hhT + (long long)k * NXh * NY;
            const float2* hn = hN + (long long)k * NY;
            __syncwarp();
#pragma unroll
            for (int mm = 0; mm < QN; ++mm) tr[lane + 32 * mm] = p[mm];
            __syncwarp();
#pragma unroll
            for (int mm = 0; mm < QN; ++mm) {
                const int f = lane + 32 * mm;
                float2 x, y;
                split_dc_nyq(p[mm], tr_partner<NY>(tr, f), x, y);
                float2 r = cmulc(x, __ldg(&h0[f]));
                const float2 s = cmulc(y, __ldg(&hn[f]));
                r.x -= s.y;
                r.y += s.x;
                p[mm] = r;
            }
            __syncwarp();
        } else {
            // V-hat times conj(hhat_k), a quarter of the column at a time (fewer
            // values live at once than a whole-column load followed by the products)
            const bool ok = use_bulk && !failed;
#pragma unroll
            for (int qq = 0; qq < NQ; ++qq) {
                float2 x[8];
                tm_load8c(t_hold + 16 * qq, x);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    p[8 * qq + j] = ok ? cmulc(x[j], tr[lane + 32 * (8 * qq + j)]) : make_float2(0.f, 0.f);
            }
        }
        // the next term's spectrum arrives while this inverse FFT finishes; at
        // the end of a slot the transpose tiles stage the store first
        const bool issue = use_bulk && !failed && kn >= 0;
        auto hook = [&] {
            if (issue && !last && lane == 0)
                bulk_load(tr, hhT + ((long long)kn * NXh + col) * NY, NY * sizeof(float2), bar, skip_copy);
        };
        // PRUNE: p[j], j < 16, are rows s_k + l + 32 j of the inverse FFT
        if constexpr (NY == kWarpN)
            warp_fft1024<true, kTmSplit, decltype(hook), false, PRUNE>(p, tr, tw, hook);
        else
            warp_fft512<true, kTmSplit, decltype(hook)>(p, tr, tw, hook);
        // this term's row factors have landed; the other buffer was last read
        // in the previous term
        cp_async_wait_all();
        __syncthreads();
        if (kn >= 0) {
            wy_load<NY>(wys + ((t + 1) & 1) * NY, sep.wrow, kn);
            cp_async_commit();
        }
        const float* wr = wys + (t & 1) * NY;
        if constexpr (PRUNE) {
            const int q0 = __ldg(&sep.kq0[k]);
            if (first) {   // the slot accumulator starts at zero on every row
                float2 z[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) z[j] = make_float2(0.f, 0.f);
#pragma unroll
                for (int qq = 0; qq < NQ; ++qq) tm_store8c(t_acc + 16 * qq, z);
                tm_wait_st();
            }
            float2 a[QN];
            tm_load16_rot(t_acc, q0, a);
#pragma unroll
            for (int j = 0; j < 16; ++j) a[j] = cadd(a[j], cscale(p[j], wr[lane + 32 * ((q0 + j) & 31)]));
            tm_store16_rot(t_acc, q0, a);
        } else if (first) {
#pragma unroll
            for (int qq = 0; qq < NQ; ++qq) {
                float2 a[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) a[j] = cscale(p[8 * qq + j], wr[lane + 32 * (8 * qq + j)]);
                tm_store8c(t_acc + 16 * qq, a);
            }
        } else {
#pragma unroll
            for (int qq = 0; qq < NQ; ++qq)
                tm_update8(t_acc, qq, [&](int mm, float2 a) { return cadd(a, cscale(p[mm], wr[lane + 32 * mm])); });
        }
        tm_wait_st();
        if (last) {
            // S_j of the slot: stage the four columns, store the slot box rows
            float2 s[QN];
            tm_loadq<QN>(t_acc, s);
#pragma unroll
            for (int mm = 0; mm < QN; ++mm) tile[4 * (lane + 32 * mm) + swl] = s[mm];
            __syncthreads();
            const Box bx = box[sl];
            store_cols<NY>(Q + b * q_bstride + sl * q_kstride, tile, bx.r0, bx.nr, NXh, col0);
            __syncthreads();   // the transpose tiles are free again
            if (issue && lane == 0)
                bulk_load(tr, hhT + ((long long)kn * NXh + col) * NY, NY * sizeof(float2), bar, skip_copy);
        }
    }
    tm_end(&tm_slot, kt_tm_cols<NY>());
}

}  // namespace pce
