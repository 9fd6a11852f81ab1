// plan.h -- the plan object and the runtime calls shared by the C ABI
// (pce_api.cu) and the batch scheduler / autotuner (batch.cu).  Internal:
// not part of include/pce.h.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "kernels.cuh"
#include "pce.h"

using pce::Box;
using pce::SecGeom;

struct pce_plan {
    int ndims = 0, ny = 1, nx = 0, m = 0;
    uint32_t flags = 0;
    int device = 0;
    // windows
    std::vector<Box> box;
    Box* d_box = nullptr;
    float* wbox = nullptr;      // 2D: box copies; 1D: dense [m][N]
    // spectra
    float2* hh = nullptr;       // 2D [m][ny][nx/2]; 1D packed [m][n/2]
    float2* hN = nullptr;       // 2D [m][ny]
    float2* hhT = nullptr;      // 2D, ny = 1024: [m][nx/2][ny] (each column's spectrum contiguous);
                                // ny = 2048: [m][nx/2][2][1024] (even, odd frequencies of each column)
    float2* tw1024 = nullptr;   // four-step twiddles when a transform length is 1024 (or 2048)
    float2* hN2 = nullptr;      // 2D, ny = 2048: Nyquist-column spectra split by parity [m][2][1024]
    void* hN2_16 = nullptr;
    float2* tw2048l = nullptr;  // W2048^l, l < 32
    int* d_status = nullptr;    // device status word (bit 0: a bounded wait gave up)
    // 1D of more than 8192 points: four-step over an l1ny x l1nx view
    bool l1 = false;
    int l1ny = 0, l1nx = 0;
    float2* twN = nullptr;      // W_N^j, j < N
    float2* hh4 = nullptr;      // [m][l1ny][l1nx]: hhat_k[a + l1ny * b] at (a, b)
    // reduced storage (PCE_FLAG_LOWP_STORAGE): bfloat16 window copies, half2 spectra / hscale[k]
    bool lowp = false;
    void* wbox16 = nullptr;
    void* hh16 = nullptr;
    void* hN16 = nullptr;
    void* hhT16 = nullptr;
    float* hscale = nullptr;
    long long wait_limit = 2000000000ll;   // clock cycles a kernel waits on an mbarrier
    int skip_copy = 0;          // test support: arm barriers without copying
    // twiddles
    float2* twx = nullptr;
    float2* twy = nullptr;
    // work lists
    int2* items = nullptr;
    int nitems = 0;
    int* kptr = nullptr;
    int* klist = nullptr;
    // scratch
    float2* scrZ = nullptr;
    float2* scrA = nullptr;
    int nrmax = 0;
    int bchunk = 1;             // right-hand sides the plan's scratch holds
    // autotuned choices (pce_plan_autotune): 0 = default
    int run_chunk = 0;          // right-hand sides per launch, <= bchunk
    int col_variant = 0;        // columns of 1024: 0 one-warp four-step, 1 radix-8 Stockham,
                                // 2 (separable plans) one-warp with the warp state in tensor memory,
                                // 3 the same with pruned column transforms (sep_prune),
                                // 4 variant 2 run slot by slot (row and column pass per slot)
    int row_variant = 0;        // adjoint row pass: 0 register prefetch, 1 none (3 CTAs per SM)
    double tuned_ms = 0.0;      // measured ms per right-hand side (forward + adjoint) / 2
    std::vector<double> tune_log;   // (chunk, col variant, row variant, ms per apply) per timed candidate
    long long zalloc = 0;   // Z scratch per right-hand side (float2)
    long long scratch_bytes = 0;
    // separable windows w_k = wy_k (x) wx_k (pce_plan_create_separable), Ny = 1024:
    // one slot of row spectra per distinct column factor
    bool sep = false;
    int nslots = 0;
    float* wrow = nullptr;      // [m][ny] row factors
    float* wxbox = nullptr;     // column factors of the slots on their column boxes
    Box* d_vbox = nullptr;      // [nslots] slot boxes (rows: union of the slot's row supports; ldw 0)
    int* d_kslot = nullptr;     // [m]
    int* d_korder = nullptr;    // [nterms] active terms grouped by slot
    int nterms = 0;
    int2* sitems = nullptr;     // F1 items of the slots
    int nsitems = 0;
    int* skptr = nullptr;       // G3 lists of the slots
    int* sklist = nullptr;
    long long zk_s = 0;         // float2 per slot (rows of the largest slot box x nx/2)
    // slot-by-slot schedule (column variant 4): slot j's F1 items are
    // sitems[slot_item_off[j] .. slot_item_off[j + 1]), its terms
    // korder[slot_term_off[j] .. slot_term_off[j + 1])
    std::vector<int> slot_item_off, slot_term_off;
    // pruned tensor-memory column kernels: every active term's row factor lies in
    // rows [32 kq0[k], 32 kq0[k] + 512) mod 1024; spectra rotated by W1024^{32 f kq0[k]}
    bool sep_prune = false;
    int* d_kq0 = nullptr;       // [m]
    float2* hhTr = nullptr;     // [m][nx/2][1024]
    float2* hNr = nullptr;      // [m][1024]
    // sectioned apply (PCE_FLAG_SECTIONED): per term a 1024 x sec_lc section
    bool sect = false;
    int sec_lc = 0;
    SecGeom* d_geo_f = nullptr;   // [nsec] forward windows
    SecGeom* d_geo_a = nullptr;   // [nsec] adjoint windows
    int2* sec_items_box = nullptr;   // (k, pair) over the box rows
    int2* sec_items_win = nullptr;   // (k, pair) over the forward output window rows
    int n_items_box = 0, n_items_win = 0;
    float2* hsT = nullptr;        // [m][sec_lc/2][1024] section spectra of h_k (c = 0: DC column)
    float2* hsN = nullptr;        // [m][1024] Nyquist column
    // reduced storage: half2 section spectra / sec_hscale[k] (FP32 copies freed)
    __half2* hsT16 = nullptr;
    __half2* hsN16 = nullptr;
    float* sec_hscale = nullptr;
    float2* sec_twc = nullptr;    // Stockham twiddles of sec_lc
    float2* scrZs = nullptr;      // [chunk][nsec][rows][sec_lc/2]
    float2* scrAs = nullptr;
    int nsec = 0;                 // sections: one per (term, column tile of its box)
    long long sec_k = 0, sec_b = 0;   // float2 per section, per right-hand side
    int sec_chunk = 1;
    // per-kernel timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;          // pairs (start, stop)
    std::vector<int> ev_kind;
    size_t ev_used = 0;

    void drop_events() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        ev.clear();
        ev_kind.clear();
        ev_used = 0;
    }

    ~pce_plan() {
        drop_events();
        void* ptrs[] = {d_box,  wbox,  hh,     hN,   hhT,   tw1024, d_status, twx, twy == twx ? nullptr : twy,
                        items,  kptr,  klist,  scrZ, scrA,  wbox16, hh16,     hN16, hhT16, hscale,
                        twN,    hh4,   wrow, wxbox, d_vbox, d_kslot, d_korder, sitems, skptr, sklist,
                        hN2,    hN2_16, tw2048l, d_geo_f, d_geo_a, sec_items_box, sec_items_win, hsT, hsN,
                        sec_twc, scrZs, scrAs, hsT16, hsN16, sec_hscale, d_kq0, hhTr, hNr};
        for (void* q : ptrs)
            if (q) cudaFree(q);
    }
};

namespace pce_rt {

// Scratch an apply runs on: Z/Q (per right-hand side zstride float2) and A/V
// (astride float2), room for `chunk` right-hand sides.
struct Scratch {
    float2* Z = nullptr;
    float2* A = nullptr;
    long long zstride = 0;
    long long astride = 0;
    int chunk = 1;
    int col_variant = -1;   // >= 0: overrides the plan's column variant for this apply
    int row_variant = -1;   // >= 0: overrides the plan's row variant for this apply
};

pce_status fail(pce_status s, const char* fmt, ...);
bool is_device_ptr(const void* p);
pce_status check_io(pce_plan_t p, const float* in, const float* out, int64_t batch);
// The plan's own scratch (with the tuned chunk).
Scratch plan_scratch(const pce_plan* p);
// float2 of Z/Q and A/V one right-hand side needs (0, 0 for 1D sizes <= 8192).
void scratch_per_rhs(const pce_plan* p, long long& zstride, long long& astride);
// Launch one apply (all chunks) on s with the given scratch; timing events
// only when allowed and s is not capturing.
pce_status apply_with(pce_plan_t p, const float* in, float* out, int64_t batch, bool adjoint,
                      cudaStream_t s, const Scratch& scr, bool allow_timing);
// Algorithmic FP32 flops of one apply of `batch` right-hand sides.
double model_flops(const pce_plan* p, int64_t batch);

}  // namespace pce_rt
