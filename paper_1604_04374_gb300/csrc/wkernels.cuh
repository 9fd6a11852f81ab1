// wkernels.cuh -- warp-FFT column kernels for columns of length Ny = 1024 and 512.
// They compute exactly what the generic column kernels of kernels.cuh
// compute, with the same global layouts (the spectra also in a transposed
// copy), but every column FFT (1024 or 512 points) is done by one warp (warpfft.cuh):
// no CTA barrier inside an FFT and one shared-memory transpose per FFT,
// where the generic kernel needs three barrier-separated exchanges.
// (For the row passes the generic kernels stay faster: they keep 48 warps
// per SM resident, the one-warp FFT's 32 elements per lane allow about 12.)
//
// One warp per half-spectrum column, 4 columns per CTA.  The
// column data are moved between global memory and the warps through a
// shared tile [row][4] whose column index is XOR-swizzled by (row >> 2) & 3
// (tix): a half-warp reading one column of 16 consecutive rows, or writing
// 4 columns of 4 rows, hits 16 distinct 8-byte bank slots.  The tile is
// filled with cp.async 8-byte copies of 32-byte row segments; the copy of the
// next term's tile overlaps the current term's FFT.
#pragma once

#include "kernels.cuh"
#include "warpfft.cuh"

namespace pce {

constexpr int kWarpN = 1024;
constexpr int kWColWarps = 4;          // columns per CTA of the column kernels
// shared memory for columns of NY points: the column tile, one NY-point
// transpose tile per warp, and two NY-float buffers of row factors (separable
// windows)
template <int NY>
constexpr int kw_col_smem() {
    return (NY * kWColWarps + kWColWarps * NY) * (int)sizeof(float2) + 2 * NY * (int)sizeof(float);
}
constexpr int kWColSmem = kw_col_smem<kWarpN>();
// resident CTAs per SM the column kernels are compiled for: 3 at 1024 points
// (168 registers), 5 at 512 points (at most 102 registers)
template <int NY>
constexpr int kw_col_min_ctas() { return NY == kWarpN ? 3 : 5; }

// element (row, column c < 4) of the swizzled column tile
__device__ __forceinline__ int tix(int row, int c) { return row * kWColWarps + (c ^ ((row >> 2) & 3)); }
// A lane touches rows r0 + 32 q: (row >> 2) & 3 is the same for all of them,
// so tix(r0 + 32 q, c) = 4 (r0 + 32 q) + sw with sw = c ^ ((r0 >> 2) & 3).
__device__ __forceinline__ int tix_sw(int r0, int c) { return c ^ ((r0 >> 2) & 3); }

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool pred) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int sz = pred ? 8 : 0;   // src-size 0: write zeros, read nothing
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ---- bulk asynchronous copies (TMA engine) tracked by an mbarrier
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Arm the barrier for `bytes` and, unless skip_copy, copy `bytes` from global
// memory to shared memory on the TMA engine.  Called by one lane.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar,
                                          bool skip_copy) {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    if (!skip_copy)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                smem_addr(dst)),
            "l"(src), "r"(bytes), "r"(smem_addr(bar))
            : "memory");
}

// Wait for phase `parity` of the barrier, for at most kWaitCycles clock
// cycles (about a second).  Returns false when the wait gave up.
constexpr long long kWaitCycles = 2000000000ll;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long limit) {
    const long long t0 = clock64();
    while (true) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// Device status word of a plan: bit 0 = a bounded wait gave up.
constexpr int kStatusTimeout = 1;

// ----------------------------------------------------------- column kernels
// Cooperative async copy of rows [0, nrows) of a [rows][nxh] column tile
// (columns col0 .. col0+3) into the shared tile, row i -> tile row i.
__device__ __forceinline__ void tile_load(float2* tile, const float2* __restrict__ src, int nrows_tile,
                                          int nxh, int col0) {
    for (int e = threadIdx.x; e < nrows_tile * kWColWarps; e += kWColWarps * 32) {
        const int i = e >> 2, c = e & 3;
        const bool ok = col0 + c < nxh;
        cp_async8(tile + tix(i, c), src + (long long)i * nxh + (ok ? col0 + c : 0), ok);
    }
    cp_async_commit();
}

// Separable windows: cooperative async copy of row factor wy_k (NY floats)
// into one of the two row-factor buffers (committed with the next group).
template <int NY = kWarpN>
__device__ __forceinline__ void wy_load(float* dst, const float* __restrict__ wrow, int k) {
    const float* src = wrow + (long long)k * NY;
    for (int e = threadIdx.x; e < NY / 4; e += kWColWarps * 32) cp_async16(dst + 4 * e, src + 4 * e);
}

// The DC/Nyquist column (column 0 of tile 0): separate the FFT of
// DC + i Nyquist at f = lane + 32 m into A (DC) and B (Nyquist).
template <int Q>
__device__ __forceinline__ void warp_split(const float2 (&v)[Q], int lane, int m, float2& A, float2& B) {
    split_dc_nyq(v[m], warp_partner(v, lane, m), A, B);
}

// F2 for Ny = NY (1024 or 512).  Grid (batch, NXh / 4), 128 threads,
// kw_col_smem<NY>() bytes.
// hhT: [m][NXh][NY] (column c's spectrum contiguous; c = 0: DC column),
// hN: [m][NY] (Nyquist column).
// SEP = false: Z holds one slot per term (box[k] rows of w_k . u's row spectra).
// SEP = true: Z holds one slot per column factor (box[] indexed by slot), each
// term's column is its slot's column times wy_k (row factor) on load, and a
// slot's tile is loaded once for all of its terms.
template <typename HT = float2, bool SEP = false, int NY = kWarpN>
__global__ void __launch_bounds__(kWColWarps * 32, kw_col_min_ctas<NY>())
kw_cols_fwd(const float2* __restrict__ Z, long long z_bstride, long long z_kstride,
            const HT* __restrict__ hhT, const HT* __restrict__ hN, const float* __restrict__ hscale, int m,
            const Box* __restrict__ box, int NXh, float2* __restrict__ A, long long a_bstride,
            const float2* __restrict__ tw, int* __restrict__ status, long long wait_limit, int skip_copy,
            SepTerms sep = SepTerms{}) {
    constexpr int QN = NY / 32;   // values per lane
    extern __shared__ float2 smem[];
    float2* tile = smem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* tr = smem + NY * kWColWarps + warp * NY;
    const int b = blockIdx.x;
    const int col0 = blockIdx.y * kWColWarps;
    const int col = col0 + warp;
    const bool cv = col < NXh;
    const bool dcn = blockIdx.y == 0 && warp == 0;
    const float2* Zb = Z + b * z_bstride;
    __shared__ unsigned long long bars[kWColWarps];
    unsigned long long* bar = &bars[warp];
    if (lane == 0) mbar_init(bar);
    __syncwarp();
    unsigned parity = 0;
    bool failed = false;

    float2 acc[QN];
#pragma unroll
    for (int i = 0; i < QN; ++i) acc[i] = make_float2(0.f, 0.f);
    // the sequence of terms: general, every term with a nonempty box in index
    // order (slot = term); separable, sep.korder (slot = sep.kslot[term])
    const int tend = SEP ? sep.nterms : m;
    auto next_t = [&](int t) {
        if constexpr (!SEP) {
            while (t < m && box[t].nr == 0) ++t;
        }
        return t;
    };
    auto kof = [&](int t) { return SEP ? __ldg(&sep.korder[t]) : t; };
    auto slot_of = [&](int kk) { return SEP ? __ldg(&sep.kslot[kk]) : kk; };
    // SEP: row factors of term t in buffer (t & 1), prefetched one term ahead
    float* wys = reinterpret_cast<float*>(smem + 2 * NY * kWColWarps);
    int t = next_t(0);
    int cur_slot = -1;
    if (t < tend) {
        const int s0 = slot_of(kof(t));
        if constexpr (SEP) wy_load<NY>(wys, sep.wrow, kof(t));
        tile_load(tile, Zb + s0 * z_kstride, box[s0].nr, NXh, col0);
    }
    while (t < tend) {
        const int k = kof(t);
        const int sl = slot_of(k);
        const int tn = next_t(t + 1);
        const int sn = tn < tend ? slot_of(kof(tn)) : -1;
        const Box bx = box[sl];
        if (SEP || sl != cur_slot) {   // uniform over the CTA
            cp_async_wait_all();
            __syncthreads();
            cur_slot = sl;
        }
        float2 v[QN];
        if constexpr (SEP) {
            const float* wr = wys + (t & 1) * NY;
            if (bx.r0 == 0 && bx.nr == NY) {   // uniform: the slot holds every row in place
                const float2* tb = tile + 4 * lane + tix_sw(lane, warp);
#pragma unroll
                for (int q = 0; q < QN; ++q) v[q] = cscale(tb[128 * q], wr[lane + 32 * q]);
            } else {
#pragma unroll
                for (int q = 0; q < QN; ++q) {
                    const int i = wrap(lane + 32 * q - bx.r0, NY);
                    v[q] = (i < bx.nr) ? cscale(tile[tix(i, warp)], wr[lane + 32 * q]) : make_float2(0.f, 0.f);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < QN; ++q) {
                const int i = wrap(lane + 32 * q - bx.r0, NY);
                v[q] = (i < bx.nr) ? tile[tix(i, warp)] : make_float2(0.f, 0.f);
            }
        }
        if (tn < tend && sn != sl) {   // the next term needs another slot: reload the tile
            __syncthreads();
            tile_load(tile, Zb + sn * z_kstride, box[sn].nr, NXh, col0);
        }
        // this column's spectrum of term k arrives in the warp's transpose
        // tile while the FFT finishes
        const bool bulk = !dcn && cv && !failed;
        const float sk = hscale_of<HT>(hscale, k);
        warp_fft<NY, false>(v, tr, tw, [&] {
            if (bulk && lane == 0)
                bulk_load(tr, hhT + ((long long)k * NXh + col) * NY, NY * sizeof(HT), bar, skip_copy);
        });
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
            const HT* h0 = hhT + (long long)k * NXh * NY;
            const HT* hn = hN + (long long)k * NY;
#pragma unroll
            for (int mm = 0; mm < QN; ++mm) {
                const int f = lane + 32 * mm;
                float2 a, bb;
                warp_split(v, lane, mm, a, bb);
                acc[mm] = cfma(ldh(&h0[f], sk), a, acc[mm]);
                const float2 t = cmul(ldh(&hn[f], sk), bb);
                acc[mm].x -= t.y;
                acc[mm].y += t.x;
            }
        } else if (cv && !failed) {
            const HT* th = reinterpret_cast<const HT*>(tr);
#pragma unroll
            for (int mm = 0; mm < QN; ++mm) acc[mm] = cfma(lds_h(&th[lane + 32 * mm], sk), v[mm], acc[mm]);
        }
        if constexpr (SEP) {
            // next term's row factors into the other buffer, last read in the
            // previous term (before this term's barrier)
            if (tn < tend) {
                wy_load<NY>(wys + ((t + 1) & 1) * NY, sep.wrow, kof(tn));
                cp_async_commit();
            }
        }
        t = tn;
    }
    warp_fft<NY, true>(acc, tr, tw);
    __syncthreads();
    const int swl = tix_sw(lane, warp);
#pragma unroll
    for (int mm = 0; mm < QN; ++mm) tile[4 * (lane + 32 * mm) + swl] = acc[mm];
    __syncthreads();
    float2* Ab = A + b * a_bstride;
    for (int e = threadIdx.x; e < NY * kWColWarps; e += kWColWarps * 32) {
        const int i = e >> 2, c = e & 3;
        if (col0 + c < NXh) Ab[(long long)i * NXh + col0 + c] = tile[tix(i, c)];
    }
}

// G1b + G2 for Ny = NY (1024 or 512; FULL: every row of Q, for the window
// gradient).
// Grid (batch, NXh / 4).
// SEP: Q receives one slot per column factor: S_j = sum over the slot's terms of
// wy_k . IFFT_y(conj(hhat_k) V), on the slot box rows (box[] indexed by slot),
// accumulated in the shared tile and stored once per slot.
template <bool FULL, typename HT = float2, bool SEP = false, int NY = kWarpN>
__global__ void __launch_bounds__(kWColWarps * 32, kw_col_min_ctas<NY>())
kw_cols_adj(const float2* __restrict__ V, long long v_bstride,
            const HT* __restrict__ hhT, const HT* __restrict__ hN, const float* __restrict__ hscale, int m,
            const Box* __restrict__ box, int NXh,
            float2* __restrict__ Q, long long q_bstride, long long q_kstride,
            const float2* __restrict__ tw, int* __restrict__ status, long long wait_limit, int skip_copy,
            SepTerms sep = SepTerms{}) {
    constexpr int QN = NY / 32;   // values per lane
    extern __shared__ float2 smem[];
    float2* tile = smem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* tr = smem + NY * kWColWarps + warp * NY;
    const int b = blockIdx.x;
    const int col0 = blockIdx.y * kWColWarps;
    const int col = col0 + warp;
    const bool cv = col < NXh;
    const bool dcn = blockIdx.y == 0 && warp == 0;
    __shared__ unsigned long long bars[kWColWarps];
    unsigned long long* bar = &bars[warp];
    if (lane == 0) mbar_init(bar);
    __syncwarp();
    unsigned parity = 0;
    bool failed = false;
    const bool use_bulk = !dcn && cv;
    // the sequence of terms (see kw_cols_fwd)
    const int tend = SEP ? sep.nterms : m;
    auto next_t = [&](int t) {
        if constexpr (!SEP) {
            while (t < m && !FULL && box[t].nr == 0) ++t;
        }
        return t;
    };
    auto kof = [&](int t) { return SEP ? __ldg(&sep.korder[t]) : t; };
    auto slot_of = [&](int kk) { return SEP ? __ldg(&sep.kslot[kk]) : kk; };

    // SEP: row factors of the t-th term in buffer (t & 1), prefetched one term ahead
    float* wys = reinterpret_cast<float*>(smem + 2 * NY * kWColWarps);
    if constexpr (SEP) {
        if (sep.nterms > 0) wy_load<NY>(wys, sep.wrow, __ldg(&sep.korder[0]));
    }
    tile_load(tile, V + b * v_bstride, NY, NXh, col0);
    cp_async_wait_all();
    __syncthreads();
    float2 vv[QN];
#pragma unroll
    for (int q = 0; q < QN; ++q) vv[q] = tile[4 * (lane + 32 * q) + tix_sw(lane, warp)];
    int t = next_t(0);
    int prev_slot = -1;
    // the spectrum of the first term arrives while the FFT of V finishes
    warp_fft<NY, false, SEP>(vv, tr, tw, [&] {
        if (use_bulk && t < tend && lane == 0)
            bulk_load(tr, hhT + ((long long)kof(t) * NXh + col) * NY, NY * sizeof(HT), bar, skip_copy);
    });
    while (t < tend) {
        const int k = kof(t);
        const int sl = slot_of(k);
        const Box bx = box[sl];
        const int tn = next_t(t + 1);
        const int kn = tn < tend ? kof(tn) : m;
        const bool first = sl != prev_slot;
        const bool last = tn >= tend || slot_of(kn) != sl;
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
        const float sk = hscale_of<HT>(hscale, k);
        if (dcn) {
            const HT* h0 = hhT + (long long)k * NXh * NY;
            const HT* hn = hN + (long long)k * NY;
#pragma unroll
            for (int mm = 0; mm < QN; ++mm) {
                const int f = lane + 32 * mm;
                float2 a, bb;
                warp_split(vv, lane, mm, a, bb);
                float2 t = cmulc(a, ldh(&h0[f], sk));
                const float2 s = cmulc(bb, ldh(&hn[f], sk));
                t.x -= s.y;
                t.y += s.x;
                p[mm] = t;
            }
        } else {
            const HT* th = reinterpret_cast<const HT*>(tr);
#pragma unroll
            for (int mm = 0; mm < QN; ++mm)
                p[mm] = (use_bulk && !failed) ? cmulc(vv[mm], lds_h(&th[lane + 32 * mm], sk))
                                              : make_float2(0.f, 0.f);
        }
        // the next term's spectrum arrives while this inverse FFT finishes
        const bool issue = use_bulk && !failed && tn < tend;
        warp_fft<NY, true, SEP>(p, tr, tw, [&] {
            if (issue && lane == 0)
                bulk_load(tr, hhT + ((long long)kn * NXh + col) * NY, NY * sizeof(HT), bar, skip_copy);
        });
        if constexpr (SEP) {
            // accumulate wy_k . p into this warp's column of the tile; the previous
            // slot's store must have finished reading the tile, and this term's
            // row factors must have landed
            cp_async_wait_all();
            __syncthreads();
            if (tn < tend) {   // the other buffer was last read in the previous term
                wy_load<NY>(wys + ((t + 1) & 1) * NY, sep.wrow, kn);
                cp_async_commit();
            }
            const float* wr = wys + (t & 1) * NY;
            float2* col = tile + tix_sw(lane, warp) + 4 * lane;
            if (first) {
#pragma unroll
                for (int mm = 0; mm < QN; ++mm) col[128 * mm] = cscale(p[mm], wr[lane + 32 * mm]);
            } else {
#pragma unroll
                for (int mm = 0; mm < QN; ++mm) col[128 * mm] = cadd(col[128 * mm], cscale(p[mm], wr[lane + 32 * mm]));
            }
            if (last) {
                __syncthreads();
                float2* Qs = Q + b * q_bstride + sl * q_kstride;
                for (int e = threadIdx.x; e < bx.nr * kWColWarps; e += kWColWarps * 32) {
                    const int i = e >> 2, c = e & 3;
                    const int g = wrap(bx.r0 + i, NY);
                    if (col0 + c < NXh) Qs[(long long)i * NXh + col0 + c] = tile[tix(g, c)];
                }
            }
        } else {
            __syncthreads();
#pragma unroll
            for (int mm = 0; mm < QN; ++mm) tile[4 * (lane + 32 * mm) + tix_sw(lane, warp)] = p[mm];
            __syncthreads();
            float2* Qk = Q + b * q_bstride + k * q_kstride;
            const int rows = FULL ? NY : bx.nr;
            for (int e = threadIdx.x; e < rows * kWColWarps; e += kWColWarps * 32) {
                const int i = e >> 2, c = e & 3;
                const int g = FULL ? i : wrap(bx.r0 + i, NY);
                if (col0 + c < NXh) Qk[(long long)i * NXh + col0 + c] = tile[tix(g, c)];
            }
        }
        t = tn;
    }
}

}  // namespace pce
