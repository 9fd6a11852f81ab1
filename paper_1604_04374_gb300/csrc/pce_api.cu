// pce_api.cu -- plan builder and C ABI (include/pce.h).
//
// The plan holds, on the device: the support box copy of every window w_k,
// the spectra hhat_k in the kernels' layout, FP32 twiddle tables generated in
// FP64, the work lists of the row passes, and the scratch intermediates of
// the 2D passes (Z/Q: per-term row spectra restricted to the box rows; A/V:
// per-right-hand-side spectra).  Applies only launch kernels.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "launch.h"
#include "pce.h"
#include "plan.h"

namespace {
thread_local std::string g_err;
}  // namespace

namespace pce_rt {

pce_status fail(pce_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace pce_rt

namespace {

using pce_rt::fail;
using pce_rt::is_device_ptr;

#define PCE_CK(call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? PCE_ERR_OOM : PCE_ERR_CUDA,      \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                   \
    } while (0)

constexpr long long kScratchBudget = 1ll << 30;   // bytes of 2D scratch a plan aims for
constexpr int kMaxChunk = 64;

bool is_pow2(long long n) { return n > 0 && (n & (n - 1)) == 0; }

// ------------------------------------------------------------ plan kernels
// Twiddle table of an N-point FFT (layout of pce::FftPlan), from FP64 sincospi.
__global__ void k_twiddles(float2* tw, int n) {
    const int L = pce::ilog2(n);
    const int nfull = L / 3, rem = L % 3;
    const int nst = nfull + (rem ? 1 : 0);
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int off = 0;
    for (int s = 1; s < nst; ++s) {
        const int rs = s < nfull ? 8 : (1 << rem);
        const int ns = 1 << (3 * s);
        const int cnt = (rs - 1) * ns;
        if (idx < off + cnt) {
            const int e = idx - off;
            const int q = e / ns + 1;
            const int k = e % ns;
            const long long len = (long long)ns * rs;
            double sn, cs;
            sincospi(-2.0 * (double)((long long)q * k) / (double)len, &sn, &cs);
            tw[idx] = make_float2((float)cs, (float)sn);
            return;
        }
        off += cnt;
    }
}

// Four-step twiddles of the one-warp 1024-point FFT: tw[p * 32 + l] = W1024^{l p} (FP64 sincospi).
__global__ void k_twiddles_1024(float2* tw) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 1024) return;
    const int p = idx >> 5, l = idx & 31;
    double sn, cs;
    sincospi(-2.0 * (double)(l * p) / 1024.0, &sn, &cs);
    tw[idx] = make_float2((float)cs, (float)sn);
}

// twN[j] = W_N^j for j < N (FP64 sincospi).
__global__ void k_twiddles_N(float2* tw, long long n) {
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= n) return;
    double sn, cs;
    sincospi(-2.0 * (double)j / (double)n, &sn, &cs);
    tw[j] = make_float2((float)cs, (float)sn);
}

// x[i] = conj(x[i]) for i < n, except every per-th element from 0 when skip0
// (slot 0 of a packed 1D half spectrum holds the real pair (X[0], X[N/2])).
__global__ void k_conj(float2* x, long long n, long long per, int skip0) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (skip0 && i % per == 0) continue;
        x[i].y = -x[i].y;
    }
}

// hhat [m][N/2+1] (natural half spectrum) -> hh4 [m][ny][nx] in the four-step
// order (f = a + ny b at (a, b)), Hermitian extension, real DC and Nyquist.
__global__ void k_from_half_l1(const float2* __restrict__ hhat, int m, int ny, int nx, float2* hh4) {
    const long long N = (long long)ny * nx;
    const long long total = (long long)m * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = i / N;
        const long long e = i % N;
        const long long a = e / nx, b = e % nx;
        const long long f = a + ny * b;
        const float2* src = hhat + k * (N / 2 + 1);
        float2 v;
        if (f == 0) v = make_float2(src[0].x, 0.f);
        else if (f == N / 2) v = make_float2(src[N / 2].x, 0.f);
        else if (f < N / 2) v = src[f];
        else v = make_float2(src[N - f].x, -src[N - f].y);
        hh4[i] = v;
    }
}

__global__ void k_to_half_l1(const float2* __restrict__ hh4, int m, int ny, int nx, float2* hhat) {
    const long long N = (long long)ny * nx;
    const long long total = (long long)m * (N / 2 + 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = i / (N / 2 + 1);
        const long long f = i % (N / 2 + 1);
        hhat[i] = hh4[k * N + (f % ny) * nx + f / ny];
    }
}

// hhT[k][c][f] = hh[k][f][c] (ny x nxh per term).
__global__ void k_transpose_hh(const float2* __restrict__ hh, int m, int ny, int nxh, float2* hhT) {
    const long long total = (long long)m * ny * nxh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i % ny);
        const long long kc = i / ny;
        const int c = (int)(kc % nxh);
        const long long k = kc / nxh;
        hhT[i] = hh[(k * ny + f) * nxh + c];
    }
}

// Spectra of the pruned separable column kernels (Ny = 1024): a term whose row
// factor lies in rows [s, s + 512), s = 32 kq0[k], is transformed rotated by s,
// and FFT(x)[f] = W1024^{f s} FFT(x rotated)[f], so the spectra carry that
// phase: out[k][c][f] = hhT[k][c][f] W1024^{(f s) mod 1024} (c < nxh) and
// outN[k][f] = hN[k][f] W1024^{(f s) mod 1024}.  Phase and product in FP64.
__global__ void k_rotate_cols(const float2* __restrict__ hhT, const float2* __restrict__ hN,
                              const int* __restrict__ kq0, int m, int nxh, float2* __restrict__ out,
                              float2* __restrict__ outN) {
    const long long n = (long long)m * (nxh + 1) * 1024;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i & 1023);
        const long long kc = i >> 10;
        const int k = (int)(kc / (nxh + 1));
        const int c = (int)(kc % (nxh + 1));   // c == nxh: the Nyquist column
        const int j = (int)(((long long)f * 32 * kq0[k]) & 1023);
        double sn, cs;
        sincospi(-2.0 * (double)j / 1024.0, &sn, &cs);
        const float2 h = c < nxh ? hhT[((long long)k * nxh + c) * 1024 + f] : hN[(long long)k * 1024 + f];
        const float2 r = make_float2((float)((double)h.x * cs - (double)h.y * sn),
                                     (float)((double)h.x * sn + (double)h.y * cs));
        if (c < nxh)
            out[((long long)k * nxh + c) * 1024 + f] = r;
        else
            outN[(long long)k * 1024 + f] = r;
    }
}

// ny = 2048: hhT[k][c][par][f'] = hh[k][2 f' + par][c], hN2[k][par][f'] = hN[k][2 f' + par]
__global__ void k_split_hh2(const float2* __restrict__ hh, const float2* __restrict__ hN, int m, int nxh,
                            float2* hhT, float2* hN2) {
    const long long total = (long long)m * nxh * 2048;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int fp = (int)(i & 1023);
        const int par = (int)((i >> 10) & 1);
        const long long kc = i >> 11;
        const int c = (int)(kc % nxh);
        const long long k = kc / nxh;
        hhT[i] = hh[(k * 2048 + 2 * fp + par) * nxh + c];
        if (c == 0) hN2[(k * 2 + par) * 1024 + fp] = hN[k * 2048 + 2 * fp + par];
    }
}

// W2048^l for l < 32 (FP64 sincospi)
__global__ void k_tw2048l(float2* tw) {
    const int l = threadIdx.x;
    if (l >= 32) return;
    double sn, cs;
    sincospi(-2.0 * l / 2048.0, &sn, &cs);
    tw[l] = make_float2((float)cs, (float)sn);
}

int twiddle_len(int n) {
    const int L = pce::ilog2(n);
    const int nfull = L / 3, rem = L % 3;
    const int nst = nfull + (rem ? 1 : 0);
    int len = 0;
    for (int s = 1; s < nst; ++s) len += ((s < nfull ? 8 : (1 << rem)) - 1) * (1 << (3 * s));
    return len;
}

// Row/column nonzero flags of every window.
__global__ void k_support(const float* __restrict__ w, int m, int ny, int nx,
                          unsigned char* rowf, unsigned char* colf) {
    const long long total = (long long)m * ny * nx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        if (w[i] != 0.f) {
            const int c = (int)(i % nx);
            const long long kr = i / nx;
            const int r = (int)(kr % ny);
            const int k = (int)(kr / ny);
            rowf[(long long)k * ny + r] = 1;
            colf[(long long)k * nx + c] = 1;
        }
    }
}

// Box copy of w_k: wbox[woff + i*ldw + cc] = w_k[(r0+i) % ny][(c0+cc) % nx] (0 beyond nc).
__global__ void k_wbox(const float* __restrict__ w, int ny, int nx, Box bx, float* wbox) {
    const long long total = (long long)bx.nr * bx.ldw;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int cc = (int)(i % bx.ldw);
        const int r = (int)(i / bx.ldw);
        float v = 0.f;
        if (cc < bx.nc) v = w[(long long)((bx.r0 + r) % ny) * nx + (bx.c0 + cc) % nx];
        wbox[bx.woff + i] = v;
    }
}

// hhat [m][ny][nxh+1] (natural) -> hh [m][ny][nxh] (column 0 = Hermitian part
// of the DC column), hN [m][ny] (Hermitian part of the Nyquist column).
__global__ void k_from_half2d(const float2* __restrict__ hhat, int m, int ny, int nxh,
                              float2* hh, float2* hN) {
    const long long total = (long long)m * ny * (nxh + 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % (nxh + 1));
        const long long kf = i / (nxh + 1);
        const int f = (int)(kf % ny);
        const int k = (int)(kf / ny);
        const float2 a = hhat[i];
        if (c > 0 && c < nxh) {
            hh[((long long)k * ny + f) * nxh + c] = a;
        } else {
            const int fm = (ny - f) & (ny - 1);
            const float2 b = hhat[((long long)k * ny + fm) * (nxh + 1) + c];
            const float2 hs = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
            if (c == 0) hh[((long long)k * ny + f) * nxh] = hs;
            else hN[(long long)k * ny + f] = hs;
        }
    }
}

__global__ void k_to_half2d(const float2* __restrict__ hh, const float2* __restrict__ hN, int m,
                            int ny, int nxh, float2* hhat) {
    const long long total = (long long)m * ny * (nxh + 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % (nxh + 1));
        const long long kf = i / (nxh + 1);
        hhat[i] = c < nxh ? hh[kf * nxh + c] : hN[kf];
    }
}

// hhat [m][n/2+1] -> packed [m][n/2] (slot 0 = (Re DC, Re Nyquist)) and back.
__global__ void k_from_half1d(const float2* __restrict__ hhat, int m, int nh, float2* hp) {
    const long long total = (long long)m * nh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i % nh);
        const long long k = i / nh;
        const float2* src = hhat + k * (nh + 1);
        hp[i] = f == 0 ? make_float2(src[0].x, src[nh].x) : src[f];
    }
}

__global__ void k_to_half1d(const float2* __restrict__ hp, int m, int nh, float2* hhat) {
    const long long total = (long long)m * (nh + 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i % (nh + 1));
        const long long k = i / (nh + 1);
        const float2* src = hp + k * nh;
        float2 v;
        if (f == 0) v = make_float2(src[0].x, 0.f);
        else if (f == nh) v = make_float2(src[0].y, 0.f);
        else v = src[f];
        hhat[i] = v;
    }
}

// ----- kernels of the plain unfused per-term pipeline (PCE_FLAG_UNFUSED)
// tmp[b] = w_k . u_b on the whole grid (zero outside w_k's box).  Grid-stride.
__global__ void k_plain_window(const float* __restrict__ u, long long P, int ny, int nx, int nb,
                               const float* __restrict__ wbox, Box bx, float* __restrict__ tmp) {
    const long long total = (long long)nb * P;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long pix = i % P;
        const int r = (int)(pix / nx), c = (int)(pix % nx);
        const int ir = pce::wrap(r - bx.r0, ny), cc = pce::wrap(c - bx.c0, nx);
        float v = 0.f;
        if (ir < bx.nr && cc < bx.nc) v = wbox[bx.woff + (long long)ir * bx.ldw + cc] * u[i];
        tmp[i] = v;
    }
}

// x[b] (+)= w_k . t[b] (whole grid).  first: overwrite instead of accumulate.
__global__ void k_plain_window_acc(const float* __restrict__ t, long long P, int ny, int nx, int nb,
                                   const float* __restrict__ wbox, Box bx, float* __restrict__ x,
                                   int first) {
    const long long total = (long long)nb * P;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long pix = i % P;
        const int r = (int)(pix / nx), c = (int)(pix % nx);
        const int ir = pce::wrap(r - bx.r0, ny), cc = pce::wrap(c - bx.c0, nx);
        float v = 0.f;
        if (ir < bx.nr && cc < bx.nc) v = wbox[bx.woff + (long long)ir * bx.ldw + cc] * t[i];
        x[i] = first ? v : x[i] + v;
    }
}

// Spectral product on the [nb][ny][nxh] (+ Nyquist [nb][ny]) layout:
// mode 0: acc += hhat_k . S ; mode 1: acc = conj(hhat_k) . S.
__global__ void k_plain_spec_mac(const float2* __restrict__ S, const float2* __restrict__ SN,
                                 const float2* __restrict__ hk, const float2* __restrict__ hNk,
                                 int ny, int nxh, int nb, float2* __restrict__ acc,
                                 float2* __restrict__ accN, int mode) {
    const long long per = (long long)ny * (nxh + 1);
    const long long total = (long long)nb * per;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / per;
        const long long e = i % per;
        const int f = (int)(e / (nxh + 1));
        const int c = (int)(e % (nxh + 1));
        float2 h, x;
        float2* dst;
        if (c < nxh) {
            h = hk[(long long)f * nxh + c];
            x = S[(b * ny + f) * nxh + c];
            dst = acc + (b * ny + f) * nxh + c;
        } else {
            h = hNk[f];
            x = SN[b * ny + f];
            dst = accN + b * ny + f;
        }
        if (mode == 0) *dst = pce::cfma(h, x, *dst);
        else *dst = pce::cmulc(x, h);
    }
}

// CTAs of the R2C row kernel for `items` row pairs of length nx.
unsigned r2c_blocks(int items, int nx) {
    const int ipc = pce::rows_r2c_items_per_cta(nx);
    return (unsigned)((items + ipc - 1) / ipc);
}

// ----- reduced storage: per-term scale, half2 spectra, bfloat16 windows
// out[k] (float bits) = max over term k's entries of max(|Re|, |Im|).
__global__ void k_term_maxabs(const float2* __restrict__ a, long long per, int m, unsigned* out) {
    const long long total = per * m;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 v = a[i];
        const float x = fmaxf(fabsf(v.x), fabsf(v.y));
        atomicMax(&out[i / per], __float_as_uint(x));   // non-negative floats order as their bits
    }
}

// dst[i] = half2(src[i] / s_k); src[i] is replaced by the value dst[i] stands for.
__global__ void k_quantize_h(float2* src, long long per, int m, const float* __restrict__ scale,
                             __half2* dst) {
    const long long total = per * m;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const float sk = scale[i / per];
        const float2 v = src[i];
        const __half2 h = __floats2half2_rn(v.x / sk, v.y / sk);
        dst[i] = h;
        const float2 f = __half22float2(h);
        src[i] = make_float2(f.x * sk, f.y * sk);
    }
}

__global__ void k_quantize_w(float* src, long long n, __nv_bfloat16* dst) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const __nv_bfloat16 b = __float2bfloat16_rn(src[i]);
        dst[i] = b;
        src[i] = __bfloat162float(b);
    }
}

unsigned grid_for(long long total, int threads = 256) {
    long long g = (total + threads - 1) / threads;
    return (unsigned)std::max<long long>(1, std::min<long long>(g, 1 << 20));
}

// Smallest periodic interval [start, start+len) holding every set flag.
void cyclic_support(const unsigned char* f, int n, int& start, int& len) {
    int nz = 0;
    for (int i = 0; i < n; ++i) nz += f[i] != 0;
    if (nz == 0) { start = 0; len = 0; return; }
    if (nz == n) { start = 0; len = n; return; }
    // longest cyclic run of zeros
    int best = 0, best_end = 0, run = 0;
    for (int t = 0; t < 2 * n; ++t) {
        if (!f[t % n]) {
            ++run;
            if (run > best && run <= n) { best = run; best_end = t; }
        } else {
            run = 0;
        }
    }
    start = (best_end + 1) % n;
    len = n - best;
}

template <class T>
pce_status dev_alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return PCE_OK;
    PCE_CK(cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T)));
    return PCE_OK;
}

}  // namespace

namespace {

// Window and spectrum storage the fused kernels read.
const void* wstore(pce_plan_t p) { return p->lowp ? p->wbox16 : (const void*)p->wbox; }
const void* hstore(pce_plan_t p) { return p->lowp ? p->hh16 : (const void*)p->hh; }
const void* hNstore(pce_plan_t p) { return p->lowp ? p->hN16 : (const void*)p->hN; }
const void* hTstore(pce_plan_t p) { return p->lowp ? p->hhT16 : (const void*)p->hhT; }
const void* hN2store(pce_plan_t p) { return p->lowp ? p->hN2_16 : (const void*)p->hN2; }

pce_status validate_shape(int ndims, const int64_t* shape, int& ny, int& nx) {
    if (ndims != 1 && ndims != 2) return fail(PCE_ERR_INVALID, "ndims must be 1 or 2 (got %d)", ndims);
    if (!shape) return fail(PCE_ERR_INVALID, "shape is NULL");
    if (ndims == 1) {
        ny = 1;
        if (!is_pow2(shape[0]) || shape[0] < 16 || shape[0] > (1 << 18))
            return fail(PCE_ERR_UNSUPPORTED, "1D size must be a power of two in [16, 262144] (got %lld)",
                        (long long)shape[0]);
        nx = (int)shape[0];
    } else {
        for (int d = 0; d < 2; ++d)
            if (!is_pow2(shape[d]) || shape[d] < 16 || shape[d] > 2048)
                return fail(PCE_ERR_UNSUPPORTED,
                            "2D sizes must be powers of two in [16, 2048] (got %lld x %lld)",
                            (long long)shape[0], (long long)shape[1]);
        ny = (int)shape[0];
        nx = (int)shape[1];
    }
    return PCE_OK;
}

pce_status make_twiddles_l1(pce_plan* p, cudaStream_t s) {
    const long long N = p->nx;
    pce_status st = dev_alloc(&p->twN, (size_t)N);
    if (st) return st;
    k_twiddles_N<<<grid_for(N), 256, 0, s>>>(p->twN, N);
    PCE_CK(cudaGetLastError());
    if ((st = dev_alloc(&p->twx, (size_t)twiddle_len(p->l1nx)))) return st;
    k_twiddles<<<grid_for(twiddle_len(p->l1nx)), 256, 0, s>>>(p->twx, p->l1nx);
    PCE_CK(cudaGetLastError());
    if (p->l1ny == p->l1nx) {
        p->twy = p->twx;
    } else {
        if ((st = dev_alloc(&p->twy, (size_t)twiddle_len(p->l1ny)))) return st;
        k_twiddles<<<grid_for(twiddle_len(p->l1ny)), 256, 0, s>>>(p->twy, p->l1ny);
        PCE_CK(cudaGetLastError());
    }
    return PCE_OK;
}

pce_status make_twiddles(pce_plan* p, cudaStream_t s) {
    if (p->l1) return make_twiddles_l1(p, s);
    // the one-warp FFTs index the 1024-point four-step table: transforms of
    // 1024, columns of 2048 (two warps per column), rows and columns of 512
    // (rows 2p of it)
    if (p->nx == 1024 || (p->ndims == 2 && (p->nx == 512 || p->ny == 512 || p->ny == 1024 || p->ny == 2048))) {
        pce_status st0 = dev_alloc(&p->tw1024, 1024);
        if (st0) return st0;
        k_twiddles_1024<<<4, 256, 0, s>>>(p->tw1024);
        PCE_CK(cudaGetLastError());
    }
    pce_status st = dev_alloc(&p->twx, (size_t)std::max(1, twiddle_len(p->nx)));
    if (st) return st;
    k_twiddles<<<grid_for(twiddle_len(p->nx)), 256, 0, s>>>(p->twx, p->nx);
    PCE_CK(cudaGetLastError());
    if (p->ndims == 2) {
        if (p->ny == p->nx) {
            p->twy = p->twx;
        } else {
            st = dev_alloc(&p->twy, (size_t)std::max(1, twiddle_len(p->ny)));
            if (st) return st;
            k_twiddles<<<grid_for(twiddle_len(p->ny)), 256, 0, s>>>(p->twy, p->ny);
            PCE_CK(cudaGetLastError());
        }
    }
    return PCE_OK;
}

// Windows: support boxes, box copies, work lists, scratch (2D); dense copy (1D).
pce_status setup_windows(pce_plan* p, const float* w, cudaStream_t s) {
    const int m = p->m, ny = p->ny, nx = p->nx;
    if (p->ndims == 1) {
        pce_status st = dev_alloc(&p->wbox, (size_t)m * nx);
        if (st) return st;
        PCE_CK(cudaMemcpyAsync(p->wbox, w, sizeof(float) * m * nx, cudaMemcpyDeviceToDevice, s));
        p->box.assign(m, Box{0, 1, 0, nx, 0, nx, 0});
        return PCE_OK;
    }
    unsigned char* flags = nullptr;
    const size_t nflags = (size_t)m * (ny + nx);
    PCE_CK(cudaMalloc(&flags, nflags));
    cudaError_t e = cudaMemsetAsync(flags, 0, nflags, s);
    if (e == cudaSuccess) {
        k_support<<<grid_for((long long)m * ny * nx), 256, 0, s>>>(w, m, ny, nx, flags,
                                                                   flags + (size_t)m * ny);
        e = cudaGetLastError();
    }
    std::vector<unsigned char> hf(nflags);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hf.data(), flags, nflags, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(flags);
    PCE_CK(e);

    p->box.resize(m);
    long long woff = 0;
    for (int k = 0; k < m; ++k) {
        Box b{};
        cyclic_support(&hf[(size_t)k * ny], ny, b.r0, b.nr);
        cyclic_support(&hf[(size_t)m * ny + (size_t)k * nx], nx, b.c0, b.nc);
        if (b.nr == 0 || b.nc == 0) { b.nr = 0; b.nc = 0; }
        b.ldw = (b.nc + 3) & ~3;
        b.woff = woff;
        woff += (long long)b.nr * b.ldw;
        p->box[k] = b;
        p->nrmax = std::max(p->nrmax, b.nr);
    }
    pce_status st = dev_alloc(&p->wbox, (size_t)std::max<long long>(woff, 4));
    if (st) return st;
    for (int k = 0; k < m; ++k) {
        const Box& b = p->box[k];
        if (b.nr == 0) continue;
        k_wbox<<<grid_for((long long)b.nr * b.ldw), 256, 0, s>>>(w + (size_t)k * ny * nx, ny, nx, b,
                                                                 p->wbox);
        PCE_CK(cudaGetLastError());
    }

    // F1 items: (k, row pair inside the box)
    std::vector<int2> items;
    for (int k = 0; k < m; ++k)
        for (int q = 0; q < (p->box[k].nr + 1) / 2; ++q) items.push_back(make_int2(k, q));
    p->nitems = (int)items.size();
    // G3 lists: terms whose box holds row 2q or 2q+1
    const int npairs = (ny + 1) / 2;
    std::vector<int> kptr(npairs + 1, 0), klist;
    for (int q = 0; q < npairs; ++q) {
        for (int k = 0; k < m; ++k) {
            const Box& b = p->box[k];
            if (b.nr == 0) continue;
            bool hit = false;
            for (int g = 2 * q; g < std::min(2 * q + 2, ny); ++g) {
                int i = g - b.r0;
                if (i < 0) i += ny;
                if (i < b.nr) hit = true;
            }
            if (hit) klist.push_back(k);
        }
        kptr[q + 1] = (int)klist.size();
    }
    if ((st = dev_alloc(&p->d_box, (size_t)m))) return st;
    if ((st = dev_alloc(&p->items, std::max<size_t>(items.size(), 1)))) return st;
    if ((st = dev_alloc(&p->kptr, kptr.size()))) return st;
    if ((st = dev_alloc(&p->klist, std::max<size_t>(klist.size(), 1)))) return st;
    PCE_CK(cudaMemcpyAsync(p->d_box, p->box.data(), sizeof(Box) * m, cudaMemcpyHostToDevice, s));
    if (!items.empty())
        PCE_CK(cudaMemcpyAsync(p->items, items.data(), sizeof(int2) * items.size(),
                               cudaMemcpyHostToDevice, s));
    PCE_CK(cudaMemcpyAsync(p->kptr, kptr.data(), sizeof(int) * kptr.size(), cudaMemcpyHostToDevice, s));
    if (!klist.empty())
        PCE_CK(cudaMemcpyAsync(p->klist, klist.data(), sizeof(int) * klist.size(),
                               cudaMemcpyHostToDevice, s));
    // the host vectors die at return: make the copies complete first
    PCE_CK(cudaStreamSynchronize(s));

    // scratch: Z/Q [bchunk][m][nrmax][nx/2], A/V [bchunk][ny][nx/2]
    const long long nxh = nx / 2;
    const long long zb = (long long)m * p->nrmax * nxh;
    const long long ab = (long long)ny * nxh;
    // the unfused pipeline keeps tmp (P floats), S, S2, acc (P/2 complex each) and two
    // Nyquist columns per right-hand side in the Z scratch
    const long long zplain = (p->flags & PCE_FLAG_UNFUSED) ? 2ll * ny * nx + 2ll * ny : 0;
    const long long zalloc = std::max(zb, zplain);
    p->zalloc = zalloc;
    const long long per_b = (zalloc + ab) * (long long)sizeof(float2);
    p->bchunk = (int)std::max<long long>(1, std::min<long long>(kMaxChunk, kScratchBudget / per_b));
    if ((st = dev_alloc(&p->scrZ, (size_t)std::max<long long>(1, zalloc * p->bchunk)))) return st;
    if ((st = dev_alloc(&p->scrA, (size_t)(ab * p->bchunk)))) return st;
    p->scratch_bytes = per_b * p->bchunk;
    return PCE_OK;
}

// Per-term power-of-two scales s_k = 2^ceil(log2 max |Re, Im|) over the
// spectra a ([m][per]) and b ([m][perb], may be NULL), into sc_dev ([m],
// allocated here).
pce_status term_scales(const float2* a, long long per, const float2* b, long long perb, int m, cudaStream_t s,
                       float** sc_dev) {
    unsigned* mx = nullptr;
    pce_status st;
    if ((st = dev_alloc(&mx, (size_t)m))) return st;
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned) * m, s);
    if (e == cudaSuccess) {
        k_term_maxabs<<<grid_for(per * m), 256, 0, s>>>(a, per, m, mx);
        if (b) k_term_maxabs<<<grid_for(perb * m), 256, 0, s>>>(b, perb, m, mx);
        e = cudaGetLastError();
    }
    std::vector<unsigned> hmx(m);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hmx.data(), mx, sizeof(unsigned) * m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(mx);
    PCE_CK(e);
    std::vector<float> sc(m);
    for (int k = 0; k < m; ++k) {
        float v;
        std::memcpy(&v, &hmx[k], sizeof v);
        int ex = 0;
        const float fr = std::frexp(v, &ex);   // v = fr * 2^ex, fr in [0.5, 1)
        sc[k] = (v > 0.f && std::isfinite(v)) ? std::ldexp(1.0f, fr == 0.5f ? ex - 1 : ex) : 1.0f;
    }
    if ((st = dev_alloc(sc_dev, (size_t)m))) return st;
    PCE_CK(cudaMemcpyAsync(*sc_dev, sc.data(), sizeof(float) * m, cudaMemcpyHostToDevice, s));
    PCE_CK(cudaStreamSynchronize(s));   // sc must outlive the copy
    return PCE_OK;
}

// Reduced storage of a plan whose FP32 windows and spectra are ready: bfloat16
// box copies of w_k, half2 spectra with per-term scale s_k = 2^ceil(log2 max |Re, Im|).
// The FP32 copies are replaced by the values the reduced ones stand for.
pce_status quantize_plan(pce_plan* p, cudaStream_t s) {
    const int m = p->m, ny = p->ny, nxh = p->nx / 2;
    const bool two_d = p->ndims == 2;
    const long long per = two_d ? (long long)ny * nxh : nxh;
    pce_status st;
    if ((st = term_scales(p->hh, per, two_d ? p->hN : nullptr, ny, m, s, &p->hscale))) return st;
    __half2* h16 = nullptr;
    if ((st = dev_alloc(&h16, (size_t)(per * m)))) return st;
    p->hh16 = h16;
    k_quantize_h<<<grid_for(per * m), 256, 0, s>>>(p->hh, per, m, p->hscale, h16);
    PCE_CK(cudaGetLastError());
    if (two_d) {
        __half2* n16 = nullptr;
        if ((st = dev_alloc(&n16, (size_t)ny * m))) return st;
        p->hN16 = n16;
        k_quantize_h<<<grid_for((long long)ny * m), 256, 0, s>>>(p->hN, ny, m, p->hscale, n16);
        PCE_CK(cudaGetLastError());
        if (p->hN2) {
            __half2* n2 = nullptr;
            if ((st = dev_alloc(&n2, (size_t)ny * m))) return st;
            p->hN2_16 = n2;
            k_quantize_h<<<grid_for((long long)ny * m), 256, 0, s>>>(p->hN2, ny, m, p->hscale, n2);
            PCE_CK(cudaGetLastError());
        }
        if (p->hhT) {
            __half2* t16 = nullptr;
            if ((st = dev_alloc(&t16, (size_t)(per * m)))) return st;
            p->hhT16 = t16;
            k_quantize_h<<<grid_for(per * m), 256, 0, s>>>(p->hhT, per, m, p->hscale, t16);
            PCE_CK(cudaGetLastError());
        }
    }
    long long nw = 0;
    if (two_d) {
        for (const Box& b : p->box) nw = std::max(nw, b.woff + (long long)b.nr * b.ldw);
    } else {
        nw = (long long)m * p->nx;
    }
    __nv_bfloat16* w16 = nullptr;
    if ((st = dev_alloc(&w16, (size_t)std::max<long long>(nw, 1)))) return st;
    p->wbox16 = w16;
    if (nw > 0) {
        k_quantize_w<<<grid_for(nw), 256, 0, s>>>(p->wbox, nw, w16);
        PCE_CK(cudaGetLastError());
    }
    p->lowp = true;
    return PCE_OK;
}

pce_status check_plan(pce_plan_t p) {
    if (!p) return fail(PCE_ERR_INVALID, "plan is NULL");
    return PCE_OK;
}

pce_status setup_sectioned(pce_plan* p, const float* h, cudaStream_t s);

pce_status create_common(pce_plan_t* out, int ndims, const int64_t* shape, int m, const float* w,
                         const float* h, bool spectra, uint32_t flags, void* stream) {
    if (!out) return fail(PCE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int ny = 1, nx = 0;
    pce_status st = validate_shape(ndims, shape, ny, nx);
    if (st) return st;
    if (m < 1) return fail(PCE_ERR_INVALID, "m must be >= 1 (got %d)", m);
    if ((flags & PCE_FLAG_SECTIONED) &&
        (ndims != 2 || spectra || (flags & (PCE_FLAG_UNFUSED | PCE_FLAG_PRODUCT_CONVOLUTION))))
        return fail(PCE_ERR_UNSUPPORTED, "PCE_FLAG_SECTIONED serves 2D convolution-product plans from h, "
                                         "fused");
    if (flags & ~(uint32_t)(PCE_FLAG_UNFUSED | PCE_FLAG_LOWP_STORAGE | PCE_FLAG_PRODUCT_CONVOLUTION |
                            PCE_FLAG_SECTIONED))
        return fail(PCE_ERR_INVALID, "unknown flag bits 0x%x", flags);
    if ((flags & PCE_FLAG_UNFUSED) && (flags & PCE_FLAG_LOWP_STORAGE))
        return fail(PCE_ERR_INVALID, "PCE_FLAG_UNFUSED runs FP32 storage only");
    if (!is_device_ptr(w)) return fail(PCE_ERR_INVALID, "w must be a device pointer");
    if (!is_device_ptr(h)) return fail(PCE_ERR_INVALID, spectra ? "hhat must be a device pointer"
                                                                : "h must be a device pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    static bool prepared[64] = {false};
    int dev = 0;
    PCE_CK(cudaGetDevice(&dev));
    if (dev < 64 && !prepared[dev]) {
        PCE_CK(pce::prepare_kernels());
        prepared[dev] = true;
    }
    pce_plan* p = new pce_plan();
    p->ndims = ndims;
    p->ny = ny;
    p->nx = nx;
    p->m = m;
    p->flags = flags;
    p->device = dev;
    auto bail = [&](pce_status e) {
        cudaStreamSynchronize(s);
        delete p;
        return e;
    };
    if (ndims == 1 && nx > 8192) {
        if (flags & PCE_FLAG_LOWP_STORAGE) {
            delete p;
            return fail(PCE_ERR_UNSUPPORTED, "reduced storage serves 1D sizes up to 8192");
        }
        p->l1 = true;
        int L = 0;
        while ((1 << L) < nx) ++L;
        p->l1ny = 1 << (L / 2);
        p->l1nx = nx / p->l1ny;
    }
    if ((st = make_twiddles(p, s))) return bail(st);
    if ((st = dev_alloc(&p->d_status, 1))) return bail(st);
    if (cudaMemsetAsync(p->d_status, 0, sizeof(int), s) != cudaSuccess)
        return bail(fail(PCE_ERR_CUDA, "status word initialisation failed"));
    if ((st = setup_windows(p, w, s))) return bail(st);
    const int nxh = nx / 2;
    if (p->l1) {
        const int npairs = (m + 1) / 2;
        const long long N = nx;
        if ((st = dev_alloc(&p->hh4, (size_t)(m * N)))) return bail(st);
        if (spectra) {
            k_from_half_l1<<<grid_for(m * N), 256, 0, s>>>(reinterpret_cast<const float2*>(h), m, p->l1ny,
                                                          p->l1nx, p->hh4);
            cudaError_t e = cudaGetLastError();
            if (e) return bail(fail(PCE_ERR_CUDA, "spectrum conversion: %s", cudaGetErrorString(e)));
        } else {
            float2* G = nullptr;
            if ((st = dev_alloc(&G, (size_t)(npairs * N)))) return bail(st);
            const int cpc = pce::l1_cols_per_cta(p->l1ny);
            cudaError_t e = pce::launch_l1_cols(p->l1ny, 1 /*pair*/, dim3(npairs, 1, (p->l1nx + cpc - 1) / cpc), s,
                                                h, 0, nullptr, m, p->l1nx, p->twN, G, p->twy);
            const int it = pce::l1_row_items(p->l1nx);
            if (e == cudaSuccess)
                e = pce::launch_l1_rows_spec(p->l1nx, dim3((p->l1ny / 2 + 1 + it - 1) / it, npairs), s, G, npairs,
                                             m, p->l1ny, p->hh4, p->twx);
            cudaError_t e2 = cudaStreamSynchronize(s);
            cudaFree(G);
            if (e == cudaSuccess) e = e2;
            if (e) return bail(fail(PCE_ERR_CUDA, "spectrum of h: %s", cudaGetErrorString(e)));
        }
        // scratch: per right-hand side npairs * N (G or Q) + N (A or V) complex
        const long long per_b = ((long long)npairs * N + N) * (long long)sizeof(float2);
        p->bchunk = (int)std::max<long long>(1, std::min<long long>(kMaxChunk, kScratchBudget / per_b));
        if ((st = dev_alloc(&p->scrZ, (size_t)(npairs * N * p->bchunk)))) return bail(st);
        if ((st = dev_alloc(&p->scrA, (size_t)(N * p->bchunk)))) return bail(st);
        p->scratch_bytes = per_b * p->bchunk;
    } else if (ndims == 1) {
        if ((st = dev_alloc(&p->hh, (size_t)m * nxh))) return bail(st);
        if (spectra) {
            k_from_half1d<<<grid_for((long long)m * nxh), 256, 0, s>>>(
                reinterpret_cast<const float2*>(h), m, nxh, p->hh);
            cudaError_t e = cudaGetLastError();
            if (e) return bail(fail(PCE_ERR_CUDA, "spectrum conversion: %s", cudaGetErrorString(e)));
        } else {
            cudaError_t e = pce::launch_spec_1d(nx, m, s, h, p->hh, p->twx);
            if (e) return bail(fail(PCE_ERR_CUDA, "spectrum of h: %s", cudaGetErrorString(e)));
        }
    } else {
        if ((st = dev_alloc(&p->hh, (size_t)m * ny * nxh))) return bail(st);
        if ((st = dev_alloc(&p->hN, (size_t)m * ny))) return bail(st);
        if (spectra) {
            k_from_half2d<<<grid_for((long long)m * ny * (nxh + 1)), 256, 0, s>>>(
                reinterpret_cast<const float2*>(h), m, ny, nxh, p->hh, p->hN);
            cudaError_t e = cudaGetLastError();
            if (e) return bail(fail(PCE_ERR_CUDA, "spectrum conversion: %s", cudaGetErrorString(e)));
        } else {
            // hhat = column FFT of the row R2C spectra of h (rows of all m terms at once)
            float2* S = nullptr;
            if ((st = dev_alloc(&S, (size_t)m * ny * nxh))) return bail(st);
            const int fpc = pce::rows_pairs_per_cta(nx);
            const int npairs = (ny + 1) / 2;
            cudaError_t e = pce::launch_rows_r2c(nx, false, dim3(r2c_blocks(npairs, nx), m), s, h,
                                                 (long long)ny * nx, ny, nullptr, false, nullptr, nullptr,
                                                 npairs, S, (long long)ny * nxh, 0, p->twx, p->tw1024);
            const int cpc = pce::cols_columns_per_cta(ny);
            if (e == cudaSuccess)
                e = pce::launch_cols_spec(ny, dim3(m, (nxh + cpc - 1) / cpc), s, S, nxh, p->hh, p->hN,
                                          p->twy);
            cudaError_t e2 = cudaStreamSynchronize(s);
            cudaFree(S);
            if (e == cudaSuccess) e = e2;
            if (e) return bail(fail(PCE_ERR_CUDA, "spectrum of h: %s", cudaGetErrorString(e)));
        }
    }
    if (flags & PCE_FLAG_PRODUCT_CONVOLUTION) {
        // sum_k w_k . (h_k * u) is the adjoint structure with the spectra of h~_k = conj(hhat_k)
        if (p->l1) {
            k_conj<<<grid_for((long long)m * nx), 256, 0, s>>>(p->hh4, (long long)m * nx, 1, 0);
        } else if (ndims == 1) {
            k_conj<<<grid_for((long long)m * nxh), 256, 0, s>>>(p->hh, (long long)m * nxh, nxh, 1);
        } else {
            k_conj<<<grid_for((long long)m * ny * nxh), 256, 0, s>>>(p->hh, (long long)m * ny * nxh, 1, 0);
            k_conj<<<grid_for((long long)m * ny), 256, 0, s>>>(p->hN, (long long)m * ny, 1, 0);
        }
        cudaError_t e1 = cudaGetLastError();
        if (e1) return bail(fail(PCE_ERR_CUDA, "spectrum conjugation: %s", cudaGetErrorString(e1)));
    }
    if (ndims == 2 && (ny == 1024 || ny == 512)) {
        if ((st = dev_alloc(&p->hhT, (size_t)m * ny * nxh))) return bail(st);
        k_transpose_hh<<<grid_for((long long)m * ny * nxh), 256, 0, s>>>(p->hh, m, ny, nxh, p->hhT);
        cudaError_t e1 = cudaGetLastError();
        if (e1) return bail(fail(PCE_ERR_CUDA, "spectrum transpose: %s", cudaGetErrorString(e1)));
    }
    if (ndims == 2 && ny == 2048) {
        // spectra of each column split by frequency parity for the two-warp column FFT
        if ((st = dev_alloc(&p->hhT, (size_t)m * ny * nxh))) return bail(st);
        if ((st = dev_alloc(&p->hN2, (size_t)m * ny))) return bail(st);
        if ((st = dev_alloc(&p->tw2048l, 32))) return bail(st);
        k_split_hh2<<<grid_for((long long)m * ny * nxh), 256, 0, s>>>(p->hh, p->hN, m, nxh, p->hhT, p->hN2);
        k_tw2048l<<<1, 32, 0, s>>>(p->tw2048l);
        cudaError_t e1 = cudaGetLastError();
        if (e1) return bail(fail(PCE_ERR_CUDA, "spectrum split: %s", cudaGetErrorString(e1)));
    }
    if ((flags & PCE_FLAG_LOWP_STORAGE) && (st = quantize_plan(p, s))) return bail(st);
    if ((flags & PCE_FLAG_SECTIONED) && (st = setup_sectioned(p, h, s))) return bail(st);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) return bail(fail(PCE_ERR_CUDA, "plan set-up: %s", cudaGetErrorString(e)));
    *out = p;
    return PCE_OK;
}

// w[k][r][c] = wy[k][r] * wx[k][c]
__global__ void k_outer(const float* __restrict__ wy, const float* __restrict__ wx, int m, int ny, int nx,
                        float* w) {
    const long long total = (long long)m * ny * nx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = i / ((long long)ny * nx);
        const long long e = i % ((long long)ny * nx);
        w[i] = wy[k * ny + e / nx] * wx[k * nx + e % nx];
    }
}

// Slots of the separable fast path: one per distinct column factor (bitwise),
// its column box, the union of its terms' row supports, the work lists of the
// row passes over the slots, and the term order grouped by slot.  Only for
// Ny = 1024 or 512 with FP32 storage; otherwise the plan keeps the general path.
pce_status setup_separable(pce_plan* p, const float* wy, const float* wx, cudaStream_t s) {
    const int m = p->m, ny = p->ny, nx = p->nx;
    if (p->ndims != 2 || (ny != 1024 && ny != 512) || p->lowp || (p->flags & PCE_FLAG_UNFUSED)) return PCE_OK;
    std::vector<float> hy((size_t)m * ny), hx((size_t)m * nx);
    PCE_CK(cudaMemcpyAsync(hy.data(), wy, sizeof(float) * hy.size(), cudaMemcpyDeviceToHost, s));
    PCE_CK(cudaMemcpyAsync(hx.data(), wx, sizeof(float) * hx.size(), cudaMemcpyDeviceToHost, s));
    PCE_CK(cudaStreamSynchronize(s));
    std::vector<int> kslot(m, -1), rep;   // rep[j]: first term of slot j
    for (int k = 0; k < m; ++k) {
        for (size_t j = 0; j < rep.size(); ++j)
            if (std::memcmp(&hx[(size_t)k * nx], &hx[(size_t)rep[j] * nx], sizeof(float) * nx) == 0) {
                kslot[k] = (int)j;
                break;
            }
        if (kslot[k] < 0) {
            kslot[k] = (int)rep.size();
            rep.push_back(k);
        }
    }
    const int ns = (int)rep.size();
    std::vector<int> korder;
    for (int j = 0; j < ns; ++j)
        for (int k = 0; k < m; ++k)
            if (kslot[k] == j && p->box[k].nr > 0) korder.push_back(k);
    std::vector<Box> vbox(ns);
    std::vector<float> wxb;
    int nrmax = 0;
    for (int j = 0; j < ns; ++j) {
        std::vector<unsigned char> rf(ny, 0), cf(nx, 0);
        for (int k : korder)
            if (kslot[k] == j)
                for (int r = 0; r < ny; ++r) rf[r] |= hy[(size_t)k * ny + r] != 0.f;
        for (int c = 0; c < nx; ++c) cf[c] = hx[(size_t)rep[j] * nx + c] != 0.f;
        Box b{};
        cyclic_support(rf.data(), ny, b.r0, b.nr);
        cyclic_support(cf.data(), nx, b.c0, b.nc);
        if (b.nr == 0 || b.nc == 0) { b.nr = 0; b.nc = 0; }
        b.ldw = 0;   // every row reads the same column factor
        b.woff = (long long)wxb.size();
        for (int i = 0; i < b.nc; ++i) wxb.push_back(hx[(size_t)rep[j] * nx + (b.c0 + i) % nx]);
        while (wxb.size() % 4) wxb.push_back(0.f);
        vbox[j] = b;
        nrmax = std::max(nrmax, b.nr);
    }
    const long long nxh = nx / 2;
    const long long zk = (long long)nrmax * nxh;
    if ((long long)ns * zk > p->zalloc) return PCE_OK;   // the general scratch does not hold the slots
    std::vector<int2> items;
    for (int j = 0; j < ns; ++j)
        for (int q = 0; q < (vbox[j].nr + 1) / 2; ++q) items.push_back(make_int2(j, q));
    const int npairs = (ny + 1) / 2;
    std::vector<int> kptr(npairs + 1, 0), klist;
    for (int q = 0; q < npairs; ++q) {
        for (int j = 0; j < ns; ++j) {
            const Box& b = vbox[j];
            if (b.nr == 0) continue;
            bool hit = false;
            for (int g = 2 * q; g < std::min(2 * q + 2, ny); ++g) {
                int i = g - b.r0;
                if (i < 0) i += ny;
                if (i < b.nr) hit = true;
            }
            if (hit) klist.push_back(j);
        }
        kptr[q + 1] = (int)klist.size();
    }
    pce_status st;
    if ((st = dev_alloc(&p->wrow, hy.size()))) return st;
    if ((st = dev_alloc(&p->wxbox, std::max<size_t>(wxb.size(), 4)))) return st;
    if ((st = dev_alloc(&p->d_vbox, (size_t)ns))) return st;
    if ((st = dev_alloc(&p->d_kslot, (size_t)m))) return st;
    if ((st = dev_alloc(&p->d_korder, std::max<size_t>(korder.size(), 1)))) return st;
    if ((st = dev_alloc(&p->sitems, std::max<size_t>(items.size(), 1)))) return st;
    if ((st = dev_alloc(&p->skptr, kptr.size()))) return st;
    if ((st = dev_alloc(&p->sklist, std::max<size_t>(klist.size(), 1)))) return st;
    PCE_CK(cudaMemcpyAsync(p->wrow, hy.data(), sizeof(float) * hy.size(), cudaMemcpyHostToDevice, s));
    if (!wxb.empty())
        PCE_CK(cudaMemcpyAsync(p->wxbox, wxb.data(), sizeof(float) * wxb.size(), cudaMemcpyHostToDevice, s));
    PCE_CK(cudaMemcpyAsync(p->d_vbox, vbox.data(), sizeof(Box) * ns, cudaMemcpyHostToDevice, s));
    PCE_CK(cudaMemcpyAsync(p->d_kslot, kslot.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
    if (!korder.empty())
        PCE_CK(cudaMemcpyAsync(p->d_korder, korder.data(), sizeof(int) * korder.size(), cudaMemcpyHostToDevice, s));
    if (!items.empty())
        PCE_CK(cudaMemcpyAsync(p->sitems, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, s));
    PCE_CK(cudaMemcpyAsync(p->skptr, kptr.data(), sizeof(int) * kptr.size(), cudaMemcpyHostToDevice, s));
    if (!klist.empty())
        PCE_CK(cudaMemcpyAsync(p->sklist, klist.data(), sizeof(int) * klist.size(), cudaMemcpyHostToDevice, s));
    // pruned column kernels (Ny = 1024): every active term's row factor inside
    // 512 rows that start on a multiple of 32 (the hats of a node grid with 4 or
    // more rows)
    std::vector<int> kq0(m, 0);
    bool prune = ny == 1024 && !korder.empty() && p->hhT != nullptr && p->hN != nullptr;
    for (int k : korder) {
        std::vector<unsigned char> rf(ny, 0);
        for (int r = 0; r < ny; ++r) rf[r] = hy[(size_t)k * ny + r] != 0.f;
        int r0 = 0, nr = 0;
        cyclic_support(rf.data(), ny, r0, nr);
        if (nr == 0 || (r0 & 31) + nr > 512) prune = false;
        kq0[k] = r0 >> 5;
    }
    if (prune) {
        if ((st = dev_alloc(&p->d_kq0, (size_t)m))) return st;
        if ((st = dev_alloc(&p->hhTr, (size_t)m * nxh * ny))) return st;
        if ((st = dev_alloc(&p->hNr, (size_t)m * ny))) return st;
        PCE_CK(cudaMemcpyAsync(p->d_kq0, kq0.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
        k_rotate_cols<<<grid_for((long long)m * (nxh + 1) * ny), 256, 0, s>>>(p->hhT, p->hN, p->d_kq0, m,
                                                                            (int)nxh, p->hhTr, p->hNr);
        PCE_CK(cudaGetLastError());
    }
    PCE_CK(cudaStreamSynchronize(s));   // the host vectors die at return
    p->slot_item_off.assign(ns + 1, 0);
    p->slot_term_off.assign(ns + 1, 0);
    for (int j = 0; j < ns; ++j) {
        p->slot_item_off[j + 1] = p->slot_item_off[j] + (vbox[j].nr + 1) / 2;
        int n = 0;
        for (int k : korder) n += kslot[k] == j;
        p->slot_term_off[j + 1] = p->slot_term_off[j] + n;
    }
    p->nslots = ns;
    p->nterms = (int)korder.size();
    p->nsitems = (int)items.size();
    p->zk_s = zk;
    p->sep = true;
    p->sep_prune = prune;
    return PCE_OK;
}

// h_k's support placed into a 1024 x lc section at its signed offsets:
// sec[k][(dr0 + i) mod 1024][(dc0 + j) mod lc] = h_k[(sr0 + i) mod ny][(sc0 + j) mod nx]
struct HSupport {
    int sr0, snr, sc0, snc;   // cyclic support of h_k in the grid
    int dr0, dc0;             // its first offsets, signed
};

__global__ void k_place_h(const float* __restrict__ h, int ny, int nx, const HSupport* __restrict__ sup, int m,
                          int lc, float* sec) {
    const long long total = (long long)m * 1024 * lc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / (1024LL * lc));
        const int e = (int)(i % (1024LL * lc));
        const int pr = e / lc, pc = e % lc;
        const HSupport sp = sup[k];
        // section position (pr, pc) holds offset (dr0 + i, dc0 + j) with i = (pr - dr0) mod 1024
        const int ii = ((pr - sp.dr0) % 1024 + 1024) % 1024;
        const int jj = ((pc - sp.dc0) % lc + lc) % lc;
        float v = 0.f;
        if (ii < sp.snr && jj < sp.snc)
            v = h[((long long)k * ny + (sp.sr0 + ii) % ny) * nx + (sp.sc0 + jj) % nx];
        sec[i] = v;
    }
}

// Sections of PCE_FLAG_SECTIONED: support of every h_k, section size, the
// section spectra of h_k, the windows of both directions, work lists, scratch.
pce_status setup_sectioned(pce_plan* p, const float* h, cudaStream_t s) {
    const int m = p->m, ny = p->ny, nx = p->nx;
    // exact support of every h_k (rows, columns)
    unsigned char* flags = nullptr;
    const size_t nflags = (size_t)m * (ny + nx);
    PCE_CK(cudaMalloc(&flags, nflags));
    cudaError_t e = cudaMemsetAsync(flags, 0, nflags, s);
    if (e == cudaSuccess) {
        k_support<<<grid_for((long long)m * ny * nx), 256, 0, s>>>(h, m, ny, nx, flags, flags + (size_t)m * ny);
        e = cudaGetLastError();
    }
    std::vector<unsigned char> hf(nflags);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hf.data(), flags, nflags, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(flags);
    PCE_CK(e);
    std::vector<HSupport> sup(m);
    int max_snc = 1;
    for (int k = 0; k < m; ++k) {
        HSupport& sp = sup[k];
        cyclic_support(&hf[(size_t)k * ny], ny, sp.sr0, sp.snr);
        cyclic_support(&hf[(size_t)m * ny + (size_t)k * nx], nx, sp.sc0, sp.snc);
        if (sp.snr == 0 || sp.snc == 0) { sp.snr = 0; sp.snc = 0; }
        sp.dr0 = sp.sr0 >= ny / 2 ? sp.sr0 - ny : sp.sr0;
        sp.dc0 = sp.sc0 >= nx / 2 ? sp.sc0 - nx : sp.sc0;
        const Box& b = p->box[k];
        if (b.nr == 0 || sp.snr == 0) continue;
        if (b.nr + sp.snr - 1 > 1024)
            return fail(PCE_ERR_UNSUPPORTED, "term %d: box rows %d + support rows %d - 1 exceed a 1024-row section",
                        k, b.nr, sp.snr);
        max_snc = std::max(max_snc, sp.snc);
    }
    if (max_snc > 2048)
        return fail(PCE_ERR_UNSUPPORTED, "support columns %d exceed a 2048-column section", max_snc);
    // Section width LC (a power of two, 16 .. 2048, at least every support's
    // width): each term's box columns are cut into tiles of LC - snc + 1
    // columns, one section each, and the LC of least modelled work is kept
    // (R2C / C2R of the input and output rows of every section, LC/2 pairs
    // of 1024-point column FFTs per section).
    auto live = [&](int k) { return p->box[k].nr > 0 && sup[k].snr > 0; };
    auto tiles = [&](int k, int w) { return (p->box[k].nc + (w - sup[k].snc)) / (w - sup[k].snc + 1); };
    int lc = 16;
    while (lc < max_snc) lc *= 2;
    double best = -1.0;
    int best_lc = lc;
    for (int w = lc; w <= 2048; w *= 2) {
        double cost = 0.0;
        for (int k = 0; k < m; ++k) {
            if (!live(k)) continue;
            const Box& b = p->box[k];
            const double rows = 2.0 * b.nr + sup[k].snr - 1;
            cost += tiles(k, w) * (rows * 2.5 * w * std::log2((double)w) + (w / 2) * 2.0 * 5.0 * 1024 * 10);
        }
        if (best < 0.0 || cost < best) {
            best = cost;
            best_lc = w;
        }
    }
    lc = best_lc;
    // windows: one section per (term, column tile)
    std::vector<SecGeom> gf, ga;
    std::vector<int2> ibox, iwin;
    int rows_max = 1;
    for (int k = 0; k < m; ++k) {
        if (!live(k)) continue;
        const Box& b = p->box[k];
        const HSupport& sp = sup[k];
        const int tw_c = lc - sp.snc + 1;   // box columns per tile
        const int wr = b.nr + sp.snr - 1;
        for (int t = 0, cs = 0; cs < b.nc; ++t, cs += tw_c) {
            const int nct = std::min(tw_c, b.nc - cs);
            SecGeom f{};
            f.r0 = b.r0;
            f.c0 = (b.c0 + cs) % nx;   // grid column of the tile's first box column
            f.woff = b.woff + cs;
            f.ldw = b.ldw;
            f.k = k;
            f.in_lo_r = 0;
            f.in_rows = b.nr;
            f.in_lo_c = 0;
            f.in_hi_c = nct - 1;
            f.out_lo_r = sp.dr0;
            f.out_rows = wr;
            f.out_lo_c = sp.dc0;
            f.out_hi_c = nct - 1 + sp.dc0 + sp.snc - 1;
            SecGeom a = f;
            a.in_lo_r = f.out_lo_r;
            a.in_rows = f.out_rows;
            a.in_lo_c = f.out_lo_c;
            a.in_hi_c = f.out_hi_c;
            a.out_lo_r = 0;
            a.out_rows = f.in_rows;
            a.out_lo_c = 0;
            a.out_hi_c = nct - 1;
            const int sidx = (int)gf.size();
            gf.push_back(f);
            ga.push_back(a);
            for (int q = 0; q < (f.in_rows + 1) / 2; ++q) ibox.push_back(make_int2(sidx, q));
            for (int q = 0; q < (wr + 1) / 2; ++q) iwin.push_back(make_int2(sidx, q));
        }
        rows_max = std::max(rows_max, wr);
    }
    const int nsec = (int)gf.size();
    pce_status st;
    // twiddles: one-warp 1024-point columns, Stockham rows of lc
    if (!p->tw1024) {
        if ((st = dev_alloc(&p->tw1024, 1024))) return st;
        k_twiddles_1024<<<4, 256, 0, s>>>(p->tw1024);
        PCE_CK(cudaGetLastError());
    }
    if ((st = dev_alloc(&p->sec_twc, (size_t)std::max(1, twiddle_len(lc))))) return st;
    k_twiddles<<<grid_for(twiddle_len(lc)), 256, 0, s>>>(p->sec_twc, lc);
    float2* twr = nullptr;   // Stockham twiddles of 1024 (the column pass of the section spectra)
    if ((st = dev_alloc(&twr, (size_t)twiddle_len(1024)))) return st;
    k_twiddles<<<grid_for(twiddle_len(1024)), 256, 0, s>>>(twr, 1024);
    PCE_CK(cudaGetLastError());
    // section spectra of h_k: place, row R2C, column FFT, transpose
    const int lch = lc / 2;
    HSupport* dsup = nullptr;
    float* sec = nullptr;
    float2* S = nullptr;
    float2* hs = nullptr;
    auto cleanup = [&]() {
        if (dsup) cudaFree(dsup);
        if (sec) cudaFree(sec);
        if (S) cudaFree(S);
        if (hs) cudaFree(hs);
        cudaFree(twr);
    };
    e = cudaMalloc(&dsup, sizeof(HSupport) * m);
    if (e == cudaSuccess) e = cudaMalloc(&sec, sizeof(float) * (size_t)m * 1024 * lc);
    if (e == cudaSuccess) e = cudaMalloc(&S, sizeof(float2) * (size_t)m * 1024 * lch);
    if (e == cudaSuccess) e = cudaMalloc(&hs, sizeof(float2) * (size_t)m * 1024 * lch);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dsup, sup.data(), sizeof(HSupport) * m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_place_h<<<grid_for((long long)m * 1024 * lc), 256, 0, s>>>(h, ny, nx, dsup, m, lc, sec);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = pce::launch_rows_r2c(lc, false, dim3(r2c_blocks(512, lc), m), s, sec, 1024LL * lc, 1024, nullptr, false,
                                 nullptr, nullptr, 512, S, 1024LL * lch, 0, p->sec_twc, p->tw1024);
    if (e == cudaSuccess && (st = dev_alloc(&p->hsN, (size_t)m * 1024)) != PCE_OK) {
        cleanup();
        return st;
    }
    const int cpc = pce::cols_columns_per_cta(1024);
    if (e == cudaSuccess)
        e = pce::launch_cols_spec(1024, dim3(m, (lch + cpc - 1) / cpc), s, S, lch, hs, p->hsN, twr);
    if (e == cudaSuccess && (st = dev_alloc(&p->hsT, (size_t)m * 1024 * lch)) != PCE_OK) {
        cleanup();
        return st;
    }
    if (e == cudaSuccess) {
        k_transpose_hh<<<grid_for((long long)m * 1024 * lch), 256, 0, s>>>(hs, m, 1024, lch, p->hsT);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return fail(PCE_ERR_CUDA, "section spectra: %s", cudaGetErrorString(e));
    // windows, work lists, scratch
    if ((st = dev_alloc(&p->d_geo_f, (size_t)std::max(nsec, 1)))) return st;
    if ((st = dev_alloc(&p->d_geo_a, (size_t)std::max(nsec, 1)))) return st;
    if ((st = dev_alloc(&p->sec_items_box, std::max<size_t>(ibox.size(), 1)))) return st;
    if ((st = dev_alloc(&p->sec_items_win, std::max<size_t>(iwin.size(), 1)))) return st;
    if (nsec > 0) {
        PCE_CK(cudaMemcpyAsync(p->d_geo_f, gf.data(), sizeof(SecGeom) * nsec, cudaMemcpyHostToDevice, s));
        PCE_CK(cudaMemcpyAsync(p->d_geo_a, ga.data(), sizeof(SecGeom) * nsec, cudaMemcpyHostToDevice, s));
    }
    if (!ibox.empty())
        PCE_CK(cudaMemcpyAsync(p->sec_items_box, ibox.data(), sizeof(int2) * ibox.size(), cudaMemcpyHostToDevice, s));
    if (!iwin.empty())
        PCE_CK(cudaMemcpyAsync(p->sec_items_win, iwin.data(), sizeof(int2) * iwin.size(), cudaMemcpyHostToDevice, s));
    PCE_CK(cudaStreamSynchronize(s));
    p->n_items_box = (int)ibox.size();
    p->n_items_win = (int)iwin.size();
    p->sec_lc = lc;
    p->nsec = nsec;
    p->sec_k = (long long)rows_max * lch;
    p->sec_b = (long long)std::max(nsec, 1) * p->sec_k;
    const long long per_b = 2 * p->sec_b * (long long)sizeof(float2);
    p->sec_chunk = (int)std::max<long long>(1, std::min<long long>(kMaxChunk, kScratchBudget / per_b));
    if ((st = dev_alloc(&p->scrZs, (size_t)(p->sec_b * p->sec_chunk)))) return st;
    if ((st = dev_alloc(&p->scrAs, (size_t)(p->sec_b * p->sec_chunk)))) return st;
    if (p->lowp) {
        // reduced storage: half2 section spectra with their own per-term scales
        const long long per = 1024LL * lch;
        if ((st = term_scales(p->hsT, per, p->hsN, 1024, m, s, &p->sec_hscale))) return st;
        if ((st = dev_alloc(&p->hsT16, (size_t)(per * m)))) return st;
        if ((st = dev_alloc(&p->hsN16, (size_t)m * 1024))) return st;
        k_quantize_h<<<grid_for(per * m), 256, 0, s>>>(p->hsT, per, m, p->sec_hscale, p->hsT16);
        k_quantize_h<<<grid_for(1024LL * m), 256, 0, s>>>(p->hsN, 1024, m, p->sec_hscale, p->hsN16);
        PCE_CK(cudaGetLastError());
        PCE_CK(cudaStreamSynchronize(s));
        cudaFree(p->hsT);
        cudaFree(p->hsN);
        p->hsT = nullptr;
        p->hsN = nullptr;
    }
    p->sect = true;
    return PCE_OK;
}

pce_status check_io(pce_plan_t p, const float* in, const float* out, int64_t batch) {
    if (batch < 0) return fail(PCE_ERR_INVALID, "batch must be >= 0");
    if (batch == 0) return PCE_OK;
    if (batch > (1ll << 31) - 1) return fail(PCE_ERR_INVALID, "batch too large");
    if (!is_device_ptr(in) || !is_device_ptr(out))
        return fail(PCE_ERR_INVALID, "input and output must be device pointers");
    const long long P = (long long)p->ny * p->nx;
    const char* a = reinterpret_cast<const char*>(in);
    const char* b = reinterpret_cast<const char*>(out);
    const long long bytes = P * batch * (long long)sizeof(float);
    if (a < b + bytes && b < a + bytes) return fail(PCE_ERR_INVALID, "input and output overlap");
    int dev = 0;
    PCE_CK(cudaGetDevice(&dev));
    if (dev != p->device) return fail(PCE_ERR_INVALID, "plan belongs to device %d, current is %d",
                                      p->device, dev);
    return PCE_OK;
}

// Z/Q and A/V float2 per right-hand side of the plan's apply.
void scratch_strides(const pce_plan* p, long long& zs, long long& as) {
    if (p->sect) {
        zs = p->sec_b;
        as = p->sec_b;
    } else if (p->l1) {
        zs = (long long)((p->m + 1) / 2) * p->nx;
        as = p->nx;
    } else if (p->ndims == 1) {
        zs = 0;
        as = 0;
    } else {
        zs = p->zalloc;
        as = (long long)p->ny * (p->nx / 2);
    }
}

pce_rt::Scratch own_scratch(const pce_plan* p) {
    pce_rt::Scratch r;
    r.Z = p->sect ? p->scrZs : p->scrZ;
    r.A = p->sect ? p->scrAs : p->scrA;
    scratch_strides(p, r.zstride, r.astride);
    if (p->sect)
        r.chunk = p->sec_chunk;
    else
        r.chunk = p->run_chunk > 0 ? std::min(p->run_chunk, p->bchunk) : p->bchunk;
    return r;
}

constexpr size_t kMaxTimed = 65536;

// Timing events are recorded only while an apply allows them (not under
// stream capture, not for the batch scheduler's lanes).
thread_local bool g_timing_ok = true;
struct TimingScope {
    bool saved;
    explicit TimingScope(bool ok) : saved(g_timing_ok) { g_timing_ok = ok; }
    ~TimingScope() { g_timing_ok = saved; }
};

bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Run one launch, bracketed by events when the plan records timings.
template <class F>
cudaError_t timed(pce_plan_t p, int kind, cudaStream_t s, F&& launch) {
    if (!p->timing || !g_timing_ok || p->ev_used >= 2 * kMaxTimed) return launch();
    if (p->ev_used + 2 > p->ev.size()) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
            p->ev.push_back(e);
        }
    }
    cudaEvent_t a = p->ev[p->ev_used], b = p->ev[p->ev_used + 1];
    cudaError_t err = cudaEventRecord(a, s);
    if (err == cudaSuccess) err = launch();
    if (err == cudaSuccess) err = cudaEventRecord(b, s);
    if (err == cudaSuccess) {
        p->ev_used += 2;
        p->ev_kind.push_back(kind);
    }
    return err;
}

// The plain unfused per-term pipeline (PCE_FLAG_UNFUSED), 2D.
pce_status apply_plain(pce_plan_t p, const float* in, float* out, int64_t batch, bool adjoint,
                       cudaStream_t s) {
    const int ny = p->ny, nx = p->nx, m = p->m, nxh = nx / 2;
    const long long P = (long long)ny * nx;
    const long long H = (long long)ny * nxh;
    const float scale = 1.0f / (float)P;
    const int fpc = pce::rows_pairs_per_cta(nx);
    const int cpc = pce::cols_columns_per_cta(ny);
    const int npairs = (ny + 1) / 2;
    const int tiles = (nxh + cpc - 1) / cpc;
    cudaError_t e = cudaSuccess;
    auto grid1 = [](long long total) { return grid_for(total, 256); };
    for (long long b0 = 0; b0 < batch && e == cudaSuccess; b0 += p->bchunk) {
        const int nb = (int)std::min<long long>(p->bchunk, batch - b0);
        const float* src = in + b0 * P;
        float* dst = out + b0 * P;
        float* tmp = reinterpret_cast<float*>(p->scrZ);
        float2* S = p->scrZ + (long long)nb * P / 2;
        float2* S2 = S + nb * H;
        float2* S2N = S2 + nb * H;
        float2* acc = S2N + (long long)nb * ny;
        float2* accN = acc + nb * H;
        if (!adjoint) {
            e = cudaMemsetAsync(acc, 0, sizeof(float2) * (size_t)nb * (H + ny), s);
            for (int k = 0; k < m && e == cudaSuccess; ++k) {
                const Box bx = p->box[k];
                if (bx.nr == 0) continue;
                e = timed(p, PCE_KERNEL_PLAIN, s, [&] {
                    k_plain_window<<<grid1(nb * P), 256, 0, s>>>(src, P, ny, nx, nb, p->wbox, bx, tmp);
                    return cudaGetLastError();
                });
                if (e == cudaSuccess)
                    e = timed(p, PCE_KERNEL_PLAIN, s, [&] {
                        return pce::launch_rows_r2c(nx, false, dim3(r2c_blocks(npairs, nx), nb), s, tmp,
                                                    P, ny, nullptr, false, nullptr, nullptr, npairs, S, H, 0,
                                                    p->twx, p->tw1024);
                    });
                if (e == cudaSuccess)
                    e = timed(p, PCE_KERNEL_PLAIN, s, [&] {
                        return pce::launch_cols_spec(ny, dim3(nb, tiles), s, S, nxh, S2, S2N, p->twy);
                    });
                if (e == cudaSuccess)
                    e = timed(p, PCE_KERNEL_PLAIN, s, [&] {
                        k_plain_spec_mac<<<grid1(nb * (H + ny)), 256, 0, s>>>(
                            S2, S2N, p->hh + (long long)k * H, p->hN + (long long)k * ny, ny, nxh, nb, acc,
                            accN, 0);
                        return cudaGetLastError();
                    });
            }
            if (e == cudaSuccess)
                e = timed(p, PCE_KERNEL_PLAIN, s, [&] {
                    return pce::launch_plain_cols_inv(ny, dim3(nb, tiles), s, acc, accN, nxh, p->scrA,
                                                      p->twy);
                });
            if (e == cudaSuccess)
                e = timed(p, PCE_KERNEL_PLAIN, s, [&] {
                    return pce::launch_rows_c2r(nx, dim3((npairs + fpc - 1) / fpc, nb), s, p->scrA, H, ny,
                                                dst, P, scale, p->twx, p->tw1024);
                });
        } else {
            e = timed(p, PCE_KERNEL_PLAIN, s, [&] {
                return pce::launch_rows_r2c(nx, false, dim3(r2c_blocks(npairs, nx), nb), s, src, P, ny,
                                            nullptr, false, nullptr, nullptr, npairs, S, H, 0, p->twx, p->tw1024);
            });
            if (e == cudaSuccess)
                e = timed(p, PCE_KERNEL_PLAIN, s, [&] {
                    return pce::launch_cols_spec(ny, dim3(nb, tiles), s, S, nxh, S2, S2N, p->twy);
                });
            bool first = true;
            for (int k = 0; k < m && e == cudaSuccess; ++k) {
                const Box bx = p->box[k];
                if (bx.nr == 0) continue;
                e = timed(p, PCE_KERNEL_PLAIN, s, [&] {
                    k_plain_spec_mac<<<grid1(nb * (H + ny)), 256, 0, s>>>(
                        S2, S2N, p->hh + (long long)k * H, p->hN + (long long)k * ny, ny, nxh, nb, acc,
                        accN, 1);
                    return cudaGetLastError();
                });
                if (e == cudaSuccess)
                    e = timed(p, PCE_KERNEL_PLAIN, s, [&] {
                        return pce::launch_plain_cols_inv(ny, dim3(nb, tiles), s, acc, accN, nxh, p->scrA,
                                                          p->twy);
                    });
                if (e == cudaSuccess)
                    e = timed(p, PCE_KERNEL_PLAIN, s, [&] {
                        return pce::launch_rows_c2r(nx, dim3((npairs + fpc - 1) / fpc, nb), s, p->scrA, H,
                                                    ny, tmp, P, scale, p->twx, p->tw1024);
                    });
                if (e == cudaSuccess)
                    e = timed(p, PCE_KERNEL_PLAIN, s, [&] {
                        k_plain_window_acc<<<grid1(nb * P), 256, 0, s>>>(tmp, P, ny, nx, nb, p->wbox,
                                                                              bx, dst, first ? 1 : 0);
                        return cudaGetLastError();
                    });
                first = false;
            }
            if (e == cudaSuccess && first) e = cudaMemsetAsync(dst, 0, sizeof(float) * (size_t)nb * P, s);
        }
    }
    if (e) return fail(PCE_ERR_CUDA, "unfused apply launch: %s", cudaGetErrorString(e));
    return PCE_OK;
}

pce_status apply_impl(pce_plan_t p, const float* in, float* out, int64_t batch, bool adjoint,
                      cudaStream_t s, const pce_rt::Scratch& scr, bool allow_timing = true) {
    TimingScope ts(allow_timing && !stream_capturing(s));
    // a product-convolution plan holds conj(hhat_k): its operator is the adjoint structure
    if (p->flags & PCE_FLAG_PRODUCT_CONVOLUTION) adjoint = !adjoint;
    // right-hand sides per launch: as many launches as the scratch chunk needs,
    // with equal shares (3 + 1 would leave the last launch with too few CTAs)
    const long long nch = (batch + scr.chunk - 1) / std::max(1, scr.chunk);
    const long long bal = nch > 0 ? (batch + nch - 1) / nch : 1;
    const int ny = p->ny, nx = p->nx, m = p->m, nxh = nx / 2;
    const long long P = (long long)ny * nx;
    const float scale = 1.0f / (float)P;
    cudaError_t e = cudaSuccess;
    if (p->l1) {
        const int NY = p->l1ny, NX = p->l1nx;
        const int npairs = (m + 1) / 2;
        const int cpc = pce::l1_cols_per_cta(NY);
        const int tiles = (NX + cpc - 1) / cpc;
        const int it = pce::l1_row_items(NX);
        const int kind = adjoint ? PCE_KERNEL_ADJ_1D : PCE_KERNEL_FWD_1D;
        for (long long b0 = 0; b0 < batch && e == cudaSuccess; b0 += bal) {
            const int nb = (int)std::min<long long>(bal, batch - b0);
            const float* src = in + b0 * P;
            float* dst = out + b0 * P;
            if (!adjoint) {
                e = timed(p, kind, s, [&] {
                    return pce::launch_l1_cols(NY, 0 /*window*/, dim3(npairs, nb, tiles), s, src, P, p->wbox, m, NX,
                                               p->twN, scr.Z, p->twy);
                });
                if (e == cudaSuccess)
                    e = timed(p, kind, s, [&] {
                        return pce::launch_l1_rows_fwd(NX, dim3((NY / 2 + 1 + it - 1) / it, nb), s, scr.Z, npairs,
                                                       p->hh4, m, NY, p->twN, scr.A, p->twx);
                    });
                if (e == cudaSuccess)
                    e = timed(p, kind, s, [&] {
                        return pce::launch_l1_cols_inv(NY, dim3(nb, tiles), s, scr.A, NX, dst, scale, p->twy);
                    });
            } else {
                e = timed(p, kind, s, [&] {
                    return pce::launch_l1_cols(NY, 2 /*one*/, dim3(1, nb, tiles), s, src, P, nullptr, m, NX, p->twN,
                                               scr.A, p->twy);
                });
                if (e == cudaSuccess)
                    e = timed(p, kind, s, [&] {
                        return pce::launch_l1_rows_adj(NX, dim3((NY + 2 * it - 1) / (2 * it), nb), s, scr.A,
                                                       npairs, p->hh4, m, NY, p->twN, scr.Z, p->twx);
                    });
                if (e == cudaSuccess)
                    e = timed(p, kind, s, [&] {
                        return pce::launch_l1_cols_adj(NY, dim3(nb, tiles), s, scr.Z, npairs, p->wbox, m, NX, dst,
                                                       scale, p->twy);
                    });
            }
        }
        if (e) return fail(PCE_ERR_CUDA, "1D apply launch: %s", cudaGetErrorString(e));
        return PCE_OK;
    }
    if (p->ndims == 1) {
        e = timed(p, adjoint ? PCE_KERNEL_ADJ_1D : PCE_KERNEL_FWD_1D, s, [&] {
            return adjoint
                ? pce::launch_adj_1d(nx, (int)batch, s, in, wstore(p), hstore(p), p->hscale, p->lowp, m, out, scale, p->twx,
                                     p->tw1024)
                : pce::launch_fwd_1d(nx, (int)batch, s, in, wstore(p), hstore(p), p->hscale, p->lowp, m, out, scale, p->twx,
                                     p->tw1024);
        });
        if (e) return fail(PCE_ERR_CUDA, "1D apply launch: %s", cudaGetErrorString(e));
        return PCE_OK;
    }
    if (p->flags & PCE_FLAG_UNFUSED) return apply_plain(p, in, out, batch, adjoint, s);
    if (p->sect) {
        // sections (Lemma 3.2): every term on 1024 x sec_lc points, added into the output
        const int lc = p->sec_lc, lch = lc / 2;
        const int fpc = pce::sec_rows_per_cta(lc);
        const int cpc = pce::cols_columns_per_cta(1024);
        const float sscale = 1.0f / (1024.0f * (float)lc);
        const long long nchs = (batch + scr.chunk - 1) / scr.chunk;
        const long long sbal = (batch + nchs - 1) / nchs;
        const pce::SecGeom* geo = adjoint ? p->d_geo_a : p->d_geo_f;
        const int2* it_in = adjoint ? p->sec_items_win : p->sec_items_box;
        const int n_in = adjoint ? p->n_items_win : p->n_items_box;
        const int2* it_out = adjoint ? p->sec_items_box : p->sec_items_win;
        const int n_out = adjoint ? p->n_items_box : p->n_items_win;
        for (long long b0 = 0; b0 < batch && e == cudaSuccess; b0 += sbal) {
            const int nb = (int)std::min<long long>(sbal, batch - b0);
            float* dst = out + b0 * P;
            e = cudaMemsetAsync(dst, 0, sizeof(float) * P * nb, s);
            const void* wst = wstore(p);
            const void* hst = p->lowp ? (const void*)p->hsT16 : (const void*)p->hsT;
            const void* hsn = p->lowp ? (const void*)p->hsN16 : (const void*)p->hsN;
            if (e == cudaSuccess && n_in > 0)
                e = timed(p, adjoint ? PCE_KERNEL_ROWS_R2C : PCE_KERNEL_ROWS_R2C_WINDOW, s, [&] {
                    return pce::launch_sec_r2c(lc, !adjoint, dim3((n_in + fpc - 1) / fpc, nb), s, in + b0 * P, P, ny,
                                               nx, wst, p->lowp, geo, it_in, n_in, scr.Z, scr.zstride, p->sec_k,
                                               p->sec_twc);
                });
            if (e == cudaSuccess && p->nsec > 0)   // no sections (every h_k or w_k zero): y = 0
                e = timed(p, adjoint ? PCE_KERNEL_COLS_ADJ : PCE_KERNEL_COLS_FWD, s, [&] {
                    return pce::launch_sec_cols(adjoint, dim3(p->nsec, (lch + cpc - 1) / cpc), s, scr.Z, scr.zstride,
                                                p->sec_k, nb, hst, hsn, p->sec_hscale, p->lowp, geo, lch, scr.A,
                                                scr.astride, p->sec_k, p->tw1024, p->d_status, p->wait_limit,
                                                p->skip_copy);
                });
            if (e == cudaSuccess && n_out > 0)
                e = timed(p, adjoint ? PCE_KERNEL_ROWS_ADJ : PCE_KERNEL_ROWS_C2R, s, [&] {
                    return pce::launch_sec_c2r(lc, adjoint, dim3((n_out + fpc - 1) / fpc, nb), s, scr.A, scr.astride,
                                               p->sec_k, geo, it_out, n_out, wst, p->lowp, dst, P, ny, nx, sscale,
                                               p->sec_twc);
                });
        }
        if (e) return fail(PCE_ERR_CUDA, "sectioned apply launch: %s", cudaGetErrorString(e));
        return PCE_OK;
    }
    const int colv = scr.col_variant >= 0 ? scr.col_variant : p->col_variant;
    const bool warp = colv != 1;
    const int rowv = scr.row_variant >= 0 ? scr.row_variant : p->row_variant;
    // separable fast path: one-warp column kernels only; variant 2 keeps the
    // per-warp column state in tensor memory
    const bool sepx = p->sep && warp;
    const bool septm = sepx && ((ny == 1024 && (colv == 2 || colv == 3 || colv == 4)) || (ny == 512 && colv == 2));
    // variant 4: row pass and column pass slot by slot, so that one slot's Z and
    // the accumulator A stay in L2 between them (slots without terms skipped)
    std::vector<int> active;
    if (septm && colv == 4)
        for (int j = 0; j < p->nslots; ++j)
            if (p->slot_term_off[j + 1] > p->slot_term_off[j]) active.push_back(j);
    const bool slotwise = active.size() > 1;
    pce::SepTerms sept;
    sept.wrow = p->wrow;
    sept.kslot = p->d_kslot;
    sept.korder = p->d_korder;
    sept.nterms = p->nterms;
    // the tensor-memory kernels; variant 3 runs the pruned ones (rotated spectra),
    // which the plan has when every term allows them
    const bool prune = colv == 3 && p->sep_prune;
    pce::SepTerms septp = sept;
    septp.kq0 = prune ? p->d_kq0 : nullptr;
    const float2* tm_hT = prune ? p->hhTr : p->hhT;
    const float2* tm_hN = prune ? p->hNr : p->hN;
    const long long zk = (long long)p->nrmax * nxh;
    const long long zb = scr.zstride;
    const long long ab = scr.astride;
    // row variant 2: the plain row transforms by the one-warp row kernels (rows of
    // 1024 or 512 points), the forward windowed pass by row pairs, the adjoint
    // rows by the block kernels without prefetch
    const bool wrows = rowv == 2 && (nx == 1024 || nx == 512) && p->tw1024 != nullptr;
    const int brv = rowv == 0 ? 0 : 1;
    const int fpc = pce::rows_pairs_per_cta(nx);
    const int cpc = pce::cols_columns_per_cta(ny);  // same for both variants
    const int npairs = (ny + 1) / 2;
    for (long long b0 = 0; b0 < batch && e == cudaSuccess; b0 += bal) {
        const int nb = (int)std::min<long long>(bal, batch - b0);
        const float* src = in + b0 * P;
        float* dst = out + b0 * P;
        if (slotwise && !adjoint) {
            for (size_t a = 0; a < active.size() && e == cudaSuccess; ++a) {
                const int j = active[a];
                const int i0 = p->slot_item_off[j], ni = p->slot_item_off[j + 1] - i0;
                pce::SepTerms sj = septp;
                sj.t0 = p->slot_term_off[j];
                sj.t1 = p->slot_term_off[j + 1];
                sj.mode = (a > 0 ? pce::kSepLoadAcc : 0) | (a + 1 == active.size() ? pce::kSepFinal : 0);
                if (ni > 0)
                    e = timed(p, PCE_KERNEL_ROWS_R2C_WINDOW, s, [&] {
                        return pce::launch_rows_r2c(nx, true, dim3(r2c_blocks(ni, nx), nb), s, src, P, ny, p->wxbox,
                                                    false, p->d_vbox, p->sitems + i0, ni, scr.Z, zb, p->zk_s, p->twx,
                                                    p->tw1024);
                    });
                if (e == cudaSuccess)
                    e = timed(p, PCE_KERNEL_COLS_FWD, s, [&] {
                        return pce::launch_cols_fwd_sep_tm(ny, dim3(nb, (nxh + cpc - 1) / cpc), s, scr.Z, zb, p->zk_s,
                                                           tm_hT, tm_hN, p->d_vbox, nxh, scr.A, ab, p->tw1024,
                                                           p->d_status, p->wait_limit, p->skip_copy, sj);
                    });
            }
            if (e == cudaSuccess)
                e = timed(p, PCE_KERNEL_ROWS_C2R, s, [&] {
                    if (wrows) return pce::launch_wrows_c2r(nx, nb, s, scr.A, ab, ny, dst, P, scale, p->tw1024);
                    return pce::launch_rows_c2r(nx, dim3((npairs + fpc - 1) / fpc, nb), s, scr.A, ab,
                                                ny, dst, P, scale, p->twx, p->tw1024);
                });
        } else if (slotwise) {
            e = timed(p, PCE_KERNEL_ROWS_R2C, s, [&] {
                if (wrows) return pce::launch_wrows_r2c(nx, nb, s, src, P, ny, scr.A, ab, p->tw1024);
                return pce::launch_rows_r2c(nx, false, dim3(r2c_blocks(npairs, nx), nb), s, src, P,
                                            ny, nullptr, false, nullptr, nullptr, npairs, scr.A, ab, 0,
                                            p->twx, p->tw1024);
            });
            for (size_t a = 0; a < active.size() && e == cudaSuccess; ++a) {
                const int j = active[a];
                pce::SepTerms sj = septp;
                sj.t0 = p->slot_term_off[j];
                sj.t1 = p->slot_term_off[j + 1];
                // the first pass stores V's column spectrum in place for the later ones
                sj.mode = a == 0 ? pce::kSepSpecOut : pce::kSepSpecIn;
                e = timed(p, PCE_KERNEL_COLS_ADJ, s, [&] {
                    return pce::launch_cols_adj_sep_tm(ny, dim3(nb, (nxh + cpc - 1) / cpc), s, scr.A, ab, tm_hT, tm_hN,
                                                       p->d_vbox, nxh, scr.Z, zb, p->zk_s, p->tw1024, p->d_status,
                                                       p->wait_limit, p->skip_copy, sj);
                });
                if (e == cudaSuccess)
                    e = timed(p, PCE_KERNEL_ROWS_ADJ, s, [&] {
                        return pce::launch_rows_adj(nx, dim3((npairs + fpc - 1) / fpc, nb), s, scr.Z, zb, p->zk_s,
                                                    ny, p->wxbox, false, p->d_vbox, p->skptr, p->sklist, dst, P,
                                                    scale, p->twx, p->tw1024, brv, j, j + 1, a > 0 ? 1 : 0);
                    });
            }
        } else if (sepx && !adjoint) {
            if (p->nsitems > 0)
                e = timed(p, PCE_KERNEL_ROWS_R2C_WINDOW, s, [&] {
                    if (rowv == 2)
                        return pce::launch_rows_r2c_pairs(nx, nb, s, src, P, ny, p->wxbox, false, p->d_vbox,
                                                          p->skptr, p->sklist, scr.Z, zb, p->zk_s, p->twx);
                    return pce::launch_rows_r2c(nx, true, dim3(r2c_blocks(p->nsitems, nx), nb), s, src, P, ny,
                                                p->wxbox, false, p->d_vbox, p->sitems, p->nsitems, scr.Z, zb,
                                                p->zk_s, p->twx, p->tw1024);
                });
            if (e == cudaSuccess)
                e = timed(p, PCE_KERNEL_COLS_FWD, s, [&] {
                    if (septm)
                        return pce::launch_cols_fwd_sep_tm(ny, dim3(nb, (nxh + cpc - 1) / cpc), s, scr.Z, zb, p->zk_s,
                                                           tm_hT, tm_hN, p->d_vbox, nxh, scr.A, ab, p->tw1024,
                                                           p->d_status, p->wait_limit, p->skip_copy, septp);
                    return pce::launch_cols_fwd_sep(ny, dim3(nb, (nxh + cpc - 1) / cpc), s, scr.Z, zb, p->zk_s,
                                                    p->hhT, p->hN, m, p->d_vbox, nxh, scr.A, ab, p->tw1024,
                                                    p->d_status, p->wait_limit, p->skip_copy, sept);
                });
            if (e == cudaSuccess)
                e = timed(p, PCE_KERNEL_ROWS_C2R, s, [&] {
                    if (wrows) return pce::launch_wrows_c2r(nx, nb, s, scr.A, ab, ny, dst, P, scale, p->tw1024);
                    return pce::launch_rows_c2r(nx, dim3((npairs + fpc - 1) / fpc, nb), s, scr.A, ab,
                                                ny, dst, P, scale, p->twx, p->tw1024);
                });
        } else if (sepx) {
            e = timed(p, PCE_KERNEL_ROWS_R2C, s, [&] {
                if (wrows) return pce::launch_wrows_r2c(nx, nb, s, src, P, ny, scr.A, ab, p->tw1024);
                return pce::launch_rows_r2c(nx, false, dim3(r2c_blocks(npairs, nx), nb), s, src, P,
                                            ny, nullptr, false, nullptr, nullptr, npairs, scr.A, ab, 0,
                                            p->twx, p->tw1024);
            });
            if (e == cudaSuccess)
                e = timed(p, PCE_KERNEL_COLS_ADJ, s, [&] {
                    if (septm)
                        return pce::launch_cols_adj_sep_tm(ny, dim3(nb, (nxh + cpc - 1) / cpc), s, scr.A, ab, tm_hT,
                                                           tm_hN, p->d_vbox, nxh, scr.Z, zb, p->zk_s, p->tw1024,
                                                           p->d_status, p->wait_limit, p->skip_copy, septp);
                    return pce::launch_cols_adj_sep(ny, dim3(nb, (nxh + cpc - 1) / cpc), s, scr.A, ab, p->hhT, p->hN,
                                                    m, p->d_vbox, nxh, scr.Z, zb, p->zk_s, p->tw1024,
                                                    p->d_status, p->wait_limit, p->skip_copy, sept);
                });
            if (e == cudaSuccess)
                e = timed(p, PCE_KERNEL_ROWS_ADJ, s, [&] {
                    return pce::launch_rows_adj(nx, dim3((npairs + fpc - 1) / fpc, nb), s, scr.Z, zb,
                                                p->zk_s, ny, p->wxbox, false, p->d_vbox, p->skptr, p->sklist,
                                                dst, P, scale, p->twx, p->tw1024, brv);
                });
        } else if (!adjoint) {
            if (p->nitems > 0)
                e = timed(p, PCE_KERNEL_ROWS_R2C_WINDOW, s, [&] {
                    if (rowv == 2)
                        return pce::launch_rows_r2c_pairs(nx, nb, s, src, P, ny, wstore(p), p->lowp, p->d_box,
                                                          p->kptr, p->klist, scr.Z, zb, zk, p->twx);
                    return pce::launch_rows_r2c(nx, true, dim3(r2c_blocks(p->nitems, nx), nb), s, src,
                                                P, ny, wstore(p), p->lowp, p->d_box, p->items, p->nitems, scr.Z,
                                                zb, zk, p->twx, p->tw1024);
                });
            if (e == cudaSuccess)
                e = timed(p, PCE_KERNEL_COLS_FWD, s, [&] {
                    return pce::launch_cols_fwd(ny, dim3(nb, (nxh + cpc - 1) / cpc), s, scr.Z, zb, zk,
                                                hstore(p), hNstore(p), p->hscale, p->lowp, m, p->d_box, nxh, scr.A, ab, p->twy, hTstore(p), p->tw1024, p->d_status, p->wait_limit, p->skip_copy, warp,
                                                hN2store(p), p->tw2048l);
                });
            if (e == cudaSuccess)
                e = timed(p, PCE_KERNEL_ROWS_C2R, s, [&] {
                    if (wrows) return pce::launch_wrows_c2r(nx, nb, s, scr.A, ab, ny, dst, P, scale, p->tw1024);
                    return pce::launch_rows_c2r(nx, dim3((npairs + fpc - 1) / fpc, nb), s, scr.A, ab,
                                                ny, dst, P, scale, p->twx, p->tw1024);
                });
        } else {
            e = timed(p, PCE_KERNEL_ROWS_R2C, s, [&] {
                if (wrows) return pce::launch_wrows_r2c(nx, nb, s, src, P, ny, scr.A, ab, p->tw1024);
                return pce::launch_rows_r2c(nx, false, dim3(r2c_blocks(npairs, nx), nb), s, src, P,
                                            ny, nullptr, false, nullptr, nullptr, npairs, scr.A, ab, 0,
                                            p->twx, p->tw1024);
            });
            if (e == cudaSuccess)
                e = timed(p, PCE_KERNEL_COLS_ADJ, s, [&] {
                    return pce::launch_cols_adj(ny, dim3(nb, (nxh + cpc - 1) / cpc), s, scr.A, ab,
                                                hstore(p), hNstore(p), p->hscale, p->lowp, m, p->d_box, nxh, scr.Z, zb, zk, p->twy, hTstore(p), p->tw1024, p->d_status, p->wait_limit, p->skip_copy, warp,
                                                hN2store(p), p->tw2048l);
                });
            if (e == cudaSuccess)
                e = timed(p, PCE_KERNEL_ROWS_ADJ, s, [&] {
                    return pce::launch_rows_adj(nx, dim3((npairs + fpc - 1) / fpc, nb), s, scr.Z, zb,
                                                zk, ny, wstore(p), p->lowp, p->d_box, p->kptr, p->klist, dst, P,
                                                scale, p->twx, p->tw1024, brv);
                });
        }
    }
    if (e) return fail(PCE_ERR_CUDA, "2D apply launch: %s", cudaGetErrorString(e));
    return PCE_OK;
}

}  // namespace

extern "C" {

pce_status pce_plan_create(pce_plan_t* out, int ndims, const int64_t* shape, int m, const float* w,
                           const float* h, uint32_t flags, void* stream) {
    return create_common(out, ndims, shape, m, w, h, false, flags, stream);
}

pce_status pce_plan_create_from_spectra(pce_plan_t* out, int ndims, const int64_t* shape, int m,
                                        const float* w, const float* hhat, uint32_t flags,
                                        void* stream) {
    return create_common(out, ndims, shape, m, w, hhat, true, flags, stream);
}

}  // extern "C"

namespace {

pce_status create_separable(pce_plan_t* out, const int64_t* shape, int m, const float* wy, const float* wx,
                            const float* h, bool spectra, uint32_t flags, void* stream) {
    if (!out) return fail(PCE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int ny = 1, nx = 0;
    pce_status st = validate_shape(2, shape, ny, nx);
    if (st) return st;
    if (m < 1) return fail(PCE_ERR_INVALID, "m must be >= 1 (got %d)", m);
    if (!is_device_ptr(wy) || !is_device_ptr(wx))
        return fail(PCE_ERR_INVALID, "wy and wx must be device pointers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* w = nullptr;
    if ((st = dev_alloc(&w, (size_t)m * ny * nx))) return st;
    k_outer<<<grid_for((long long)m * ny * nx), 256, 0, s>>>(wy, wx, m, ny, nx, w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFree(w);
        return fail(PCE_ERR_CUDA, "window outer products: %s", cudaGetErrorString(e));
    }
    st = create_common(out, 2, shape, m, w, h, spectra, flags, stream);
    cudaFree(w);
    if (st) return st;
    if ((st = setup_separable(*out, wy, wx, s))) {
        delete *out;
        *out = nullptr;
        return st;
    }
    return PCE_OK;
}

}  // namespace

extern "C" {

pce_status pce_plan_create_separable(pce_plan_t* out, const int64_t* shape, int m, const float* wy,
                                     const float* wx, const float* h, uint32_t flags, void* stream) {
    return create_separable(out, shape, m, wy, wx, h, false, flags, stream);
}

pce_status pce_plan_create_separable_from_spectra(pce_plan_t* out, const int64_t* shape, int m,
                                                  const float* wy, const float* wx, const float* hhat,
                                                  uint32_t flags, void* stream) {
    return create_separable(out, shape, m, wy, wx, hhat, true, flags, stream);
}

int pce_plan_slots(pce_plan_t plan) { return (plan && plan->sep) ? plan->nslots : 0; }

pce_status pce_apply(pce_plan_t plan, const float* u, float* y, int64_t batch, void* stream) {
    pce_status st = check_plan(plan);
    if (st) return st;
    if ((st = check_io(plan, u, y, batch))) return st;
    if (batch == 0) return PCE_OK;
    return apply_impl(plan, u, y, batch, false, static_cast<cudaStream_t>(stream), own_scratch(plan));
}

pce_status pce_apply_adjoint(pce_plan_t plan, const float* v, float* x, int64_t batch,
                             void* stream) {
    pce_status st = check_plan(plan);
    if (st) return st;
    if ((st = check_io(plan, v, x, batch))) return st;
    if (batch == 0) return PCE_OK;
    return apply_impl(plan, v, x, batch, true, static_cast<cudaStream_t>(stream), own_scratch(plan));
}

pce_status pce_plan_info(pce_plan_t plan, int* m_out, int* box_out, int64_t* scratch_bytes_out) {
    pce_status st = check_plan(plan);
    if (st) return st;
    if (m_out) *m_out = plan->m;
    if (box_out)
        for (int k = 0; k < plan->m; ++k) {
            box_out[4 * k + 0] = plan->box[k].r0;
            box_out[4 * k + 1] = plan->box[k].nr;
            box_out[4 * k + 2] = plan->box[k].c0;
            box_out[4 * k + 3] = plan->box[k].nc;
        }
    if (scratch_bytes_out) *scratch_bytes_out = plan->scratch_bytes;
    return PCE_OK;
}

pce_status pce_plan_hhat(pce_plan_t plan, float* hhat, void* stream) {
    pce_status st = check_plan(plan);
    if (st) return st;
    if (!is_device_ptr(hhat)) return fail(PCE_ERR_INVALID, "hhat must be a device pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nxh = plan->nx / 2;
    if (plan->l1)
        k_to_half_l1<<<grid_for((long long)plan->m * (nxh + 1)), 256, 0, s>>>(
            plan->hh4, plan->m, plan->l1ny, plan->l1nx, reinterpret_cast<float2*>(hhat));
    else if (plan->ndims == 1)
        k_to_half1d<<<grid_for((long long)plan->m * (nxh + 1)), 256, 0, s>>>(
            plan->hh, plan->m, nxh, reinterpret_cast<float2*>(hhat));
    else
        k_to_half2d<<<grid_for((long long)plan->m * plan->ny * (nxh + 1)), 256, 0, s>>>(
            plan->hh, plan->hN, plan->m, plan->ny, nxh, reinterpret_cast<float2*>(hhat));
    if (plan->flags & PCE_FLAG_PRODUCT_CONVOLUTION) {
        const long long n = (long long)plan->m * plan->ny * (nxh + 1);
        k_conj<<<grid_for(n), 256, 0, s>>>(reinterpret_cast<float2*>(hhat), n, 1, 0);
    }
    PCE_CK(cudaGetLastError());
    return PCE_OK;
}

pce_status pce_plan_destroy(pce_plan_t plan) {
    if (!plan) return PCE_OK;
    cudaError_t e = cudaDeviceSynchronize();
    delete plan;
    if (e != cudaSuccess) return fail(PCE_ERR_CUDA, "synchronise before free: %s", cudaGetErrorString(e));
    return PCE_OK;
}

const char* pce_last_error_string(void) { return g_err.c_str(); }

pce_status pce_plan_status(pce_plan_t plan, void* stream) {
    pce_status st = check_plan(plan);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int h = 0;
    PCE_CK(cudaMemcpyAsync(&h, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    PCE_CK(cudaStreamSynchronize(s));
    if (h) {
        PCE_CK(cudaMemsetAsync(plan->d_status, 0, sizeof(int), s));
        PCE_CK(cudaStreamSynchronize(s));
        return fail(PCE_ERR_TIMEOUT, "a kernel gave up a bounded wait on an asynchronous copy");
    }
    return PCE_OK;
}

pce_status pce_plan_inject_wait_timeout(pce_plan_t plan, int64_t wait_cycles) {
    pce_status st = check_plan(plan);
    if (st) return st;
    if (wait_cycles < 0) return fail(PCE_ERR_INVALID, "wait_cycles must be >= 0");
    plan->skip_copy = wait_cycles > 0 ? 1 : 0;
    plan->wait_limit = wait_cycles > 0 ? (long long)wait_cycles : 2000000000ll;
    return PCE_OK;
}

pce_status pce_plan_set_timing(pce_plan_t plan, int enable) {
    pce_status st = check_plan(plan);
    if (st) return st;
    if (!enable || plan->timing) {
        // a pending record must finish before its events are destroyed
        for (size_t i = 0; i < plan->ev_used; ++i) cudaEventSynchronize(plan->ev[i]);
        plan->drop_events();
    }
    plan->timing = enable != 0;
    return PCE_OK;
}

pce_status pce_plan_timing(pce_plan_t plan, int kind, double* total_ms, int64_t* launches) {
    pce_status st = check_plan(plan);
    if (st) return st;
    if (kind < 0 || kind >= PCE_KERNEL_KINDS) return fail(PCE_ERR_INVALID, "bad kernel kind %d", kind);
    double tot = 0.0;
    int64_t n = 0;
    for (size_t i = 0; i < plan->ev_kind.size(); ++i) {
        if (plan->ev_kind[i] != kind) continue;
        PCE_CK(cudaEventSynchronize(plan->ev[2 * i + 1]));
        float ms = 0.f;
        PCE_CK(cudaEventElapsedTime(&ms, plan->ev[2 * i], plan->ev[2 * i + 1]));
        tot += ms;
        ++n;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = n;
    return PCE_OK;
}

int64_t pce_launch_count(pce_plan_t plan, int adjoint, int64_t batch) {
    if (!plan || batch <= 0) return 0;
    if (plan->flags & PCE_FLAG_PRODUCT_CONVOLUTION) adjoint = !adjoint;
    const int64_t c = own_scratch(plan).chunk;
    const int64_t chunks = (batch + c - 1) / c;
    if (plan->l1) return chunks * 3;
    if (plan->sect) return plan->nsec > 0 ? chunks * 3 : 0;
    if (plan->ndims == 1) return 1;
    if (plan->flags & PCE_FLAG_UNFUSED) {
        int64_t mk = 0;
        for (const Box& b : plan->box) mk += b.nr > 0;
        return chunks * (4 * mk + 2);
    }
    const int64_t per = (!adjoint && plan->nitems == 0) ? 2 : 3;
    return chunks * per;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Gradients.
namespace {

constexpr long long kBackwardBudget = 2ll << 30;   // bytes of workspace per call at most

// Right-hand sides per chunk of the 2D backward and workspace float2 per right-hand side.
void backward_layout(pce_plan_t p, int64_t batch, long long& per_b, long long& chunk) {
    const long long nxh = p->nx / 2;
    const long long H = (long long)p->ny * nxh;
    per_b = 2 * H + p->ny + (long long)p->m * p->nrmax * nxh + (long long)p->m * H;
    chunk = std::max<long long>(1, std::min<long long>(batch, kBackwardBudget / (per_b * 8)));
}

}  // namespace

extern "C" int64_t pce_backward_workspace_bytes(pce_plan_t p, int64_t batch) {
    if (!p || batch < 0) return 0;
    if (p->ndims == 1) {
        // stand-in outputs for a skipped dw or dhhat
        return (int64_t)p->m * ((p->nx / 2 + 1) * 8 + p->nx * 4);
    }
    if (batch == 0) return 0;
    long long per_b, chunk;
    backward_layout(p, batch, per_b, chunk);
    return chunk * per_b * 8;
}

extern "C" pce_status pce_backward(pce_plan_t p, const float* u, const float* r, float* du, float* dw,
                                   float* dhhat, int64_t batch, void* workspace,
                                   int64_t workspace_bytes, void* stream) {
    pce_status st = check_plan(p);
    if (st) return st;
    if (batch < 0) return fail(PCE_ERR_INVALID, "batch must be >= 0");
    if (p->lowp) return fail(PCE_ERR_UNSUPPORTED, "pce_backward runs on plans with FP32 storage only");
    if (p->flags & PCE_FLAG_PRODUCT_CONVOLUTION)
        return fail(PCE_ERR_UNSUPPORTED, "pce_backward serves convolution-product plans only");
    if (p->l1) return fail(PCE_ERR_UNSUPPORTED, "pce_backward serves 1D sizes up to 8192");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int ny = p->ny, nx = p->nx, m = p->m, nxh = nx / 2;
    const long long P = (long long)ny * nx;
    const long long H = (long long)ny * nxh;
    const size_t dh_bytes = sizeof(float2) * (size_t)m * (p->ndims == 1 ? (nxh + 1) : ny * (nxh + 1));
    const size_t dw_bytes = sizeof(float) * (size_t)m * P;
    for (const void* q : {(const void*)du, (const void*)dw, (const void*)dhhat})
        if (q && !is_device_ptr(q)) return fail(PCE_ERR_INVALID, "gradient outputs must be device pointers");
    if (batch == 0) {
        if (dw) PCE_CK(cudaMemsetAsync(dw, 0, dw_bytes, s));
        if (dhhat) PCE_CK(cudaMemsetAsync(dhhat, 0, dh_bytes, s));
        return PCE_OK;
    }
    if (!is_device_ptr(u) || !is_device_ptr(r)) return fail(PCE_ERR_INVALID, "u and r must be device pointers");
    const int64_t need = pce_backward_workspace_bytes(p, batch);
    if (need > 0 && (!workspace || workspace_bytes < need || !is_device_ptr(workspace)))
        return fail(PCE_ERR_INVALID, "workspace must be a device buffer of at least %lld bytes",
                    (long long)need);
    if (du) {
        if ((st = check_io(p, r, du, batch))) return st;
        if ((st = apply_impl(p, r, du, batch, true, s, own_scratch(p)))) return st;
    }
    if (!dw && !dhhat) return PCE_OK;
    const float scale = 1.0f / (float)P;
    cudaError_t e = cudaSuccess;
    if (p->ndims == 1) {
        char* ws = static_cast<char*>(workspace);
        float2* dh_out = dhhat ? reinterpret_cast<float2*>(dhhat) : reinterpret_cast<float2*>(ws);
        float* dw_out = dw ? dw : reinterpret_cast<float*>(ws + (size_t)m * (nxh + 1) * 8);
        e = pce::launch_grad_1d(nx, m, s, u, r, p->wbox, p->hh, (int)batch, dh_out, dw_out, scale, 0, p->twx);
        if (e) return fail(PCE_ERR_CUDA, "1D backward launch: %s", cudaGetErrorString(e));
        return PCE_OK;
    }
    long long per_b, chunk;
    backward_layout(p, batch, per_b, chunk);
    const int gpc = pce::rows_grad_pairs_per_cta(nx);
    const int cpc = pce::cols_columns_per_cta(ny);
    const int npairs = (ny + 1) / 2;
    const int tiles = (nxh + cpc - 1) / cpc;
    const long long zk = (long long)p->nrmax * nxh;
    const long long zb = (long long)m * zk;
    for (long long b0 = 0; b0 < batch && e == cudaSuccess; b0 += chunk) {
        const int nb = (int)std::min<long long>(chunk, batch - b0);
        float2* S = static_cast<float2*>(workspace);
        float2* Rh = S + nb * H;
        float2* RhN = Rh + nb * H;
        float2* Zg = RhN + (long long)nb * ny;
        float2* Qf = Zg + nb * zb;
        const float* ub = u + b0 * P;
        const float* rb = r + b0 * P;
        const int acc = b0 > 0 ? 1 : 0;
        e = pce::launch_rows_r2c(nx, false, dim3(r2c_blocks(npairs, nx), nb), s, rb, P, ny, nullptr, false,
                                 nullptr, nullptr, npairs, S, H, 0, p->twx, p->tw1024);
        if (dhhat && e == cudaSuccess) {
            e = pce::launch_cols_spec(ny, dim3(nb, tiles), s, S, nxh, Rh, RhN, p->twy);
            if (e == cudaSuccess && p->nitems > 0)
                e = pce::launch_rows_r2c(nx, true, dim3(r2c_blocks(p->nitems, nx), nb), s, ub, P, ny,
                                         p->wbox, false, p->d_box, p->items, p->nitems, Zg, zb, zk, p->twx, p->tw1024);
            if (e == cudaSuccess)
                e = pce::launch_cols_grad_h(ny, dim3(m, tiles), s, Zg, zb, zk, nb, Rh, RhN, p->d_box, nxh,
                                            reinterpret_cast<float2*>(dhhat), scale, acc, p->twy);
        }
        if (dw && e == cudaSuccess) {
            e = pce::launch_cols_adj_full(ny, dim3(nb, tiles), s, S, H, p->hh, p->hN, m, p->d_box, nxh, Qf,
                                          (long long)m * H, H, p->twy, p->hhT, p->tw1024, p->d_status, p->wait_limit, p->skip_copy);
            if (e == cudaSuccess)
                e = pce::launch_rows_grad_w(nx, dim3((npairs + gpc - 1) / gpc, m), s, Qf, (long long)m * H, H,
                                            ny, nb, ub, P, dw, scale, acc, p->twx);
        }
    }
    if (e) return fail(PCE_ERR_CUDA, "2D backward launch: %s", cudaGetErrorString(e));
    return PCE_OK;
}

// ---------------------------------------------------------------------------
// Forward apply without any allocation (no counterpart in the paper).
//
// pce_apply runs the 2D passes on intermediates that the plan allocated with
// cudaMalloc.  pce_apply_noalloc runs the same three kernels on intermediates
// held in g_noalloc_scratch, a fixed array of device memory that exists as
// soon as the library is loaded on a device, so the call itself never
// allocates.  Host code may not pass g_noalloc_scratch to a kernel directly:
// in host code the name denotes a host-side shadow, not device memory.  Its
// device address comes from cudaGetSymbolAddress on the current device.
namespace {

constexpr size_t kNoallocScratchBytes = 64ull << 20;   // 64 MiB per device

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of the static scratch on the current device.  Looked up on
// every call: the lookup allocates nothing and queues no work, and a device
// reset between calls (which reloads the module, possibly elsewhere) then
// cannot leave a stale address behind.  The first lookup on a device loads
// the library's device code there if lazy loading has not done so yet.
pce_status noalloc_scratch(float2** out) {
    int dev = 0;
    PCE_CK(cudaGetDevice(&dev));
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
        return fail(PCE_ERR_CUDA, "cudaGetSymbolAddress of the static scratch on device %d: %s", dev,
                    cudaGetErrorString(e));
    *out = static_cast<float2*>(p);
    return PCE_OK;
}

}  // namespace

extern "C" pce_status pce_apply_noalloc(pce_plan_t plan, const float* u, float* y, int64_t batch,
                                        void* stream) {
    pce_status st = check_plan(plan);
    if (st) return st;
    if (plan->flags & PCE_FLAG_PRODUCT_CONVOLUTION)
        return fail(PCE_ERR_UNSUPPORTED, "pce_apply_noalloc serves convolution-product plans only");
    if (plan->ndims != 2)
        return fail(PCE_ERR_UNSUPPORTED, "pce_apply_noalloc serves 2D plans only (the 1D apply uses no scratch)");
    if ((st = check_io(plan, u, y, batch))) return st;
    if (batch == 0) return PCE_OK;
    const int ny = plan->ny, nx = plan->nx, m = plan->m, nxh = nx / 2;
    const long long zk = (long long)plan->nrmax * nxh;
    const long long zb = (long long)m * zk;
    const long long ab = (long long)ny * nxh;
    const long long per_b = (zb + ab) * (long long)sizeof(float2);
    if (per_b > (long long)kNoallocScratchBytes)
        return fail(PCE_ERR_UNSUPPORTED,
                    "pce_apply_noalloc: this plan needs %lld bytes of scratch per right-hand side, "
                    "more than the %llu bytes of static scratch",
                    per_b, (unsigned long long)kNoallocScratchBytes);
    float2* base = nullptr;
    if ((st = noalloc_scratch(&base))) return st;
    const int chunk = (int)std::min<long long>(kNoallocScratchBytes / per_b, 65535);
    float2* scrZ = base;
    float2* scrA = base + zb * chunk;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long P = (long long)ny * nx;
    const float scale = 1.0f / (float)P;
    const int fpc = pce::rows_pairs_per_cta(nx);
    const int cpc = pce::cols_columns_per_cta(ny);
    const int npairs = (ny + 1) / 2;
    cudaError_t e = cudaSuccess;
    // Every scratch element a kernel reads is written earlier in the same call
    // (Z rows inside the boxes by the row pass, all of A by the column pass),
    // so nothing left by a previous call needs clearing.
    for (long long b0 = 0; b0 < batch && e == cudaSuccess; b0 += chunk) {
        const int nb = (int)std::min<long long>(chunk, batch - b0);
        if (plan->nitems > 0)
            e = pce::launch_rows_r2c(nx, true, dim3(r2c_blocks(plan->nitems, nx), nb), s, u + b0 * P, P,
                                     ny, wstore(plan), plan->lowp, plan->d_box, plan->items, plan->nitems, scrZ, zb, zk,
                                     plan->twx, plan->tw1024);
        if (e == cudaSuccess)
            e = pce::launch_cols_fwd(ny, dim3(nb, (nxh + cpc - 1) / cpc), s, scrZ, zb, zk, hstore(plan),
                                     hNstore(plan), plan->hscale, plan->lowp, m, plan->d_box, nxh, scrA, ab,
                                     plan->twy, hTstore(plan), plan->tw1024, plan->d_status, plan->wait_limit,
                                     plan->skip_copy, plan->col_variant != 1, hN2store(plan), plan->tw2048l);
        if (e == cudaSuccess)
            e = pce::launch_rows_c2r(nx, dim3((npairs + fpc - 1) / fpc, nb), s, scrA, ab, ny, y + b0 * P, P,
                                     scale, plan->twx, plan->tw1024);
    }
    if (e) return fail(PCE_ERR_CUDA, "pce_apply_noalloc launch: %s", cudaGetErrorString(e));
    return PCE_OK;
}

// ----- runtime calls shared with the batch scheduler and the autotuner
namespace pce_rt {

pce_status check_io(pce_plan_t p, const float* in, const float* out, int64_t batch) {
    return ::check_io(p, in, out, batch);
}

Scratch plan_scratch(const pce_plan* p) { return own_scratch(p); }

void scratch_per_rhs(const pce_plan* p, long long& zstride, long long& astride) {
    scratch_strides(p, zstride, astride);
}

pce_status apply_with(pce_plan_t p, const float* in, float* out, int64_t batch, bool adjoint,
                      cudaStream_t s, const Scratch& scr, bool allow_timing) {
    return apply_impl(p, in, out, batch, adjoint, s, scr, allow_timing);
}

// Algorithmic FP32 flops of one apply: 5 n log2 n per complex FFT of n points
// (2.5 n log2 n for a real one), 8 flops per complex product-accumulate, one
// multiply per window sample.
double model_flops(const pce_plan* p, int64_t batch) {
    auto lg = [](double n) { return std::log2(n); };
    const double m = p->m;
    if (p->ndims == 1) {
        const double n = p->nx;
        return (double)batch * ((m + 1.0) * 2.5 * n * lg(n) + 8.0 * m * (n / 2 + 1) + m * n);
    }
    const double ny = p->ny, nx = p->nx, nxh1 = nx / 2 + 1;
    double rows = 0.0, win = 0.0;
    for (const Box& b : p->box) {
        rows += (double)b.nr * 2.5 * nx * lg(nx);
        win += (double)b.nr * b.nc;
    }
    const double cols = (m + 1.0) * nxh1 * 5.0 * ny * lg(ny);
    const double mac = 8.0 * m * ny * nxh1;
    const double inv = ny * 2.5 * nx * lg(nx);
    return (double)batch * (rows + win + cols + mac + inv);
}

}  // namespace pce_rt
