// launch.h -- size-dispatching launchers for the kernels in kernels.cuh.
// Every launcher picks the template instance for its transform length and
// returns the launch status (cudaGetLastError after the launch).
#pragma once

#include <cuda_runtime.h>

namespace pce {

struct Box;
struct SepTerms;
struct SecGeom;

// Shared-memory bytes and threads of the column kernels for a column length.
int cols_threads(int ny);
int cols_columns_per_cta(int ny);
int cols_smem(int ny);
// Rows handled per CTA of the row kernels (two rows per FFT).
int rows_pairs_per_cta(int nx);
// Row pairs per CTA of the window-gradient row kernel.
int rows_grad_pairs_per_cta(int nx);
// Items (row pairs) handled per CTA of the R2C row kernel.
int rows_r2c_items_per_cta(int nx);
// 1D kernels.
int fft1d_threads(int n);
int fft1d_smem(int n);

// Raise the dynamic shared-memory limit of every kernel that needs it (once per device).
cudaError_t prepare_kernels();

// Storage-precision arguments: `lowp` selects bfloat16 windows (wbox) and
// half2 spectra scaled by hscale[k]; otherwise float windows and float2 spectra.
cudaError_t launch_rows_r2c(int nx, bool window, dim3 grid, cudaStream_t s,
                            const float* src, long long src_bstride, int nrows,
                            const void* wbox, bool lowp, const Box* box, const int2* items, int nitems,
                            float2* dst, long long dst_bstride, long long dst_kstride,
                            const float2* tw, const float2* tw1024);

// F1 by row pairs (k_rows_r2c_pairs): the same output as launch_rows_r2c with a
// window, the terms (or slots) of each row pair from the CSR lists kptr/klist.
cudaError_t launch_rows_r2c_pairs(int nx, int nb, cudaStream_t s, const float* src, long long src_bstride,
                                  int nrows, const void* wbox, bool lowp, const Box* box, const int* kptr,
                                  const int* klist, float2* dst, long long dst_bstride, long long dst_kstride,
                                  const float2* tw);

cudaError_t launch_rows_c2r(int nx, dim3 grid, cudaStream_t s, const float2* src,
                            long long src_bstride, int nrows, float* dst, long long dst_bstride,
                            float scale, const float2* tw, const float2* tw1024);

cudaError_t launch_rows_adj(int nx, dim3 grid, cudaStream_t s, const float2* Q, long long q_bstride,
                            long long q_kstride, int nrows, const void* wbox, bool lowp, const Box* box,
                            const int* kptr, const int* klist, float* dst, long long dst_bstride,
                            float scale, const float2* tw, const float2* tw1024, int rv = 0, int kmin = 0,
                            int kmax = 1 << 30, int accumulate = 0);

// One-warp plain row transforms for Nx = 1024 or 512 (wrows.cuh): the same results
// and layouts as launch_rows_r2c without a window (row pairs of every row) and
// launch_rows_c2r; one warp per row pair, grids derived from nrows.
cudaError_t launch_wrows_r2c(int nx, int nb, cudaStream_t s, const float* src, long long src_bstride, int nrows,
                             float2* dst, long long dst_bstride, const float2* tw1024);
cudaError_t launch_wrows_c2r(int nx, int nb, cudaStream_t s, const float2* src, long long src_bstride, int nrows, float* dst,
                             long long dst_bstride, float scale, const float2* tw1024);

cudaError_t launch_cols_fwd(int ny, dim3 grid, cudaStream_t s, const float2* Z, long long z_bstride,
                            long long z_kstride, const void* hh, const void* hN, const float* hscale,
                            bool lowp, int m,
                            const Box* box, int nxh, float2* A, long long a_bstride,
                            const float2* tw, const void* hhT, const float2* tw1024, int* status,
                            long long wait_limit, int skip_copy, bool warp = true,
                            const void* hN2 = nullptr, const float2* tw2048l = nullptr);

cudaError_t launch_cols_adj(int ny, dim3 grid, cudaStream_t s, const float2* V, long long v_bstride,
                            const void* hh, const void* hN, const float* hscale, bool lowp, int m,
                            const Box* box, int nxh, float2* Q, long long q_bstride, long long q_kstride,
                            const float2* tw, const void* hhT, const float2* tw1024, int* status,
                            long long wait_limit, int skip_copy, bool warp = true,
                            const void* hN2 = nullptr, const float2* tw2048l = nullptr);

cudaError_t launch_cols_spec(int ny, dim3 grid, cudaStream_t s, const float2* S, int nxh,
                             float2* hh, float2* hN, const float2* tw);

cudaError_t launch_plain_cols_inv(int ny, dim3 grid, cudaStream_t s, const float2* acc,
                                  const float2* accN, int nxh, float2* A, const float2* tw);

// Sectioned apply (section.cuh)
int sec_rows_per_cta(int lc);
cudaError_t prepare_sec();
// wbox: float or bfloat16 (lowp) box copies; hsT / hsN: float2 or half2 (lowp)
// section spectra with per-term scales hscale (lowp only).
cudaError_t launch_sec_r2c(int lc, bool win, dim3 grid, cudaStream_t s, const float* src, long long src_bstride,
                           int nyg, int nxg, const void* wbox, bool lowp, const SecGeom* geo, const int2* items,
                           int nitems, float2* dst, long long dst_bstride, long long dst_kstride, const float2* tw);
cudaError_t launch_sec_cols(bool conj, dim3 grid, cudaStream_t s, const float2* Z, long long z_bstride,
                            long long z_kstride, int nb, const void* hsT, const void* hsN, const float* hscale,
                            bool lowp, const SecGeom* geo, int nxh, float2* A, long long a_bstride,
                            long long a_kstride, const float2* tw1024, int* status, long long wait_limit,
                            int skip_copy);
cudaError_t launch_sec_c2r(int lc, bool win, dim3 grid, cudaStream_t s, const float2* src, long long src_bstride,
                           long long src_kstride, const SecGeom* geo, const int2* items, int nitems,
                           const void* wbox, bool lowp, float* dst, long long dst_bstride, int nyg, int nxg,
                           float scale, const float2* tw);

// Separable windows, Ny = 1024 or 512 (one-warp column kernels): Z / Q hold
// one slot per column factor, box[] is indexed by slot.
cudaError_t launch_cols_fwd_sep(int ny, dim3 grid, cudaStream_t s, const float2* Z, long long z_bstride,
                                long long z_kstride, const float2* hhT, const float2* hN, int m,
                                const Box* box, int nxh, float2* A, long long a_bstride,
                                const float2* tw1024, int* status, long long wait_limit, int skip_copy,
                                const SepTerms& sep);
cudaError_t launch_cols_adj_sep(int ny, dim3 grid, cudaStream_t s, const float2* V, long long v_bstride,
                                const float2* hhT, const float2* hN, int m, const Box* box, int nxh,
                                float2* Q, long long q_bstride, long long q_kstride,
                                const float2* tw1024, int* status, long long wait_limit, int skip_copy,
                                const SepTerms& sep);

// The same with the per-warp state in tensor memory (tkernels.cuh), Ny = 1024 or
// 512.  With sep.kq0 set (Ny = 1024 only), the pruned kernels run and hhT / hN
// must be the rotated spectra hhat_k[f] W1024^{32 f kq0[k]}.
cudaError_t launch_cols_fwd_sep_tm(int ny, dim3 grid, cudaStream_t s, const float2* Z, long long z_bstride,
                                   long long z_kstride, const float2* hhT, const float2* hN, const Box* box,
                                   int nxh, float2* A, long long a_bstride, const float2* tw1024, int* status,
                                   long long wait_limit, int skip_copy, const SepTerms& sep);
cudaError_t launch_cols_adj_sep_tm(int ny, dim3 grid, cudaStream_t s, float2* V, long long v_bstride,
                                   const float2* hhT, const float2* hN, const Box* box, int nxh, float2* Q,
                                   long long q_bstride, long long q_kstride, const float2* tw1024, int* status,
                                   long long wait_limit, int skip_copy, const SepTerms& sep);

cudaError_t launch_cols_adj_full(int ny, dim3 grid, cudaStream_t s, const float2* V, long long v_bstride,
                                 const float2* hh, const float2* hN, int m, const Box* box, int nxh,
                                 float2* Q, long long q_bstride, long long q_kstride,
                                 const float2* tw, const float2* hhT, const float2* tw1024, int* status,
                                 long long wait_limit, int skip_copy);

cudaError_t launch_cols_grad_h(int ny, dim3 grid, cudaStream_t s, const float2* Z, long long z_bstride,
                               long long z_kstride, int nb, const float2* Rh, const float2* RhN,
                               const Box* box, int nxh, float2* dhh, float scale, int accumulate,
                               const float2* tw);

cudaError_t launch_rows_grad_w(int nx, dim3 grid, cudaStream_t s, const float2* Qf, long long q_bstride,
                               long long q_kstride, int nrows, int nb, const float* u,
                               long long u_bstride, float* dw, float scale, int accumulate,
                               const float2* tw);

cudaError_t launch_grad_1d(int n, int m, cudaStream_t s, const float* u, const float* r,
                           const float* w, const float2* hp, int nb, float2* dh, float* dw,
                           float scale, int accumulate, const float2* tw);

// tw1024 (may be NULL): the four-step table of the one-warp 1024-point FFT;
// with it, N = 1024 and fewer than 304 right-hand sides run the one-warp kernels
cudaError_t launch_fwd_1d(int n, int batch, cudaStream_t s, const float* u, const void* w,
                          const void* hp, const float* hscale, bool lowp, int m, float* y, float scale,
                          const float2* tw, const float2* tw1024 = nullptr);

cudaError_t launch_adj_1d(int n, int batch, cudaStream_t s, const float* v, const void* w,
                          const void* hp, const float* hscale, bool lowp, int m, float* x, float scale,
                          const float2* tw, const float2* tw1024 = nullptr);

cudaError_t launch_spec_1d(int n, int m, cudaStream_t s, const float* h, float2* hp,
                           const float2* tw);

// 1D transforms of N = ny * nx > 8192 points (four-step, k1d_large.cuh).
int l1_cols_per_cta(int ny);
int l1_row_items(int nx);
cudaError_t launch_l1_cols(int ny, int mode, dim3 grid, cudaStream_t s, const float* src,
                           long long src_bstride, const float* w, int m, int nx, const float2* twN,
                           float2* G, const float2* tw);
cudaError_t launch_l1_rows_fwd(int nx, dim3 grid, cudaStream_t s, const float2* G, int npairs,
                               const float2* hh4, int m, int ny, const float2* twN, float2* A,
                               const float2* tw);
cudaError_t launch_l1_cols_inv(int ny, dim3 grid, cudaStream_t s, const float2* A, int nx, float* y,
                               float scale, const float2* tw);
cudaError_t launch_l1_rows_adj(int nx, dim3 grid, cudaStream_t s, const float2* V, int npairs,
                               const float2* hh4, int m, int ny, const float2* twN, float2* Q,
                               const float2* tw);
cudaError_t launch_l1_cols_adj(int ny, dim3 grid, cudaStream_t s, const float2* Q, int npairs,
                               const float* w, int m, int nx, float* x, float scale, const float2* tw);
cudaError_t launch_l1_rows_spec(int nx, dim3 grid, cudaStream_t s, const float2* G, int npairs, int m,
                                int ny, float2* hh4, const float2* tw);

}  // namespace pce
