// tmem.cuh -- tensor memory (TMEM) as per-warp storage beside the register file.
//
// Each SM of sm_103a has 256 KB of tensor memory: 128 lanes x 512 columns of
// 32 bits.  A warp reaches only the lane quarter 32 (w % 4) .. 32 (w % 4) + 31,
// and thread i of the warp only lane 32 (w % 4) + i.  The column kernels below
// use it as 64 + 64 extra 32-bit "registers" per thread that do not count
// against the register file: the FFT input a warp reuses across terms, and the
// spectral accumulator.  Nothing here uses the tensor cores.
//
// Address format (PTX ISA, tcgen05): bits 31..16 lane, bits 15..0 column.
// An allocation is made by one warp (tcgen05.alloc writes the base address to
// shared memory), released by the same warp (tcgen05.dealloc), and covers a
// power of two of columns >= 32.  The fences order tcgen05 operations
// against the CTA barrier that publishes the address or ends its use.
#pragma once

namespace pce {

__device__ __forceinline__ void tm_alloc(unsigned* slot, int ncols) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(s), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(unsigned taddr, int ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// Wait until every tcgen05.st of this thread has completed (before the same
// columns are loaded again).
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// Loads include the wait for their completion in the same asm statement, so
// the compiler cannot move a use of the loaded registers above the wait.
// Thread i of the warp reads (writes) lane (taddr >> 16) + i, columns
// (taddr & 0xffff) .. + N - 1.
__device__ __forceinline__ void tm_ld64(unsigned taddr, unsigned (&r)[64]) {
    asm volatile(
        "{\n tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];\n"
        " tcgen05.wait::ld.sync.aligned;\n}\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tm_ld16(unsigned taddr, unsigned (&r)[16]) {
    asm volatile(
        "{\n tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
        " tcgen05.wait::ld.sync.aligned;\n}\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tm_st64(unsigned taddr, const unsigned (&r)[64]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x64.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63, %64};\n"
                 :
                 : "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31]), "r"(r[32]), "r"(r[33]), "r"(r[34]), "r"(r[35]), "r"(r[36]), "r"(r[37]), "r"(r[38]), "r"(r[39]), "r"(r[40]), "r"(r[41]), "r"(r[42]), "r"(r[43]), "r"(r[44]), "r"(r[45]), "r"(r[46]), "r"(r[47]), "r"(r[48]), "r"(r[49]), "r"(r[50]), "r"(r[51]), "r"(r[52]), "r"(r[53]), "r"(r[54]), "r"(r[55]), "r"(r[56]), "r"(r[57]), "r"(r[58]), "r"(r[59]), "r"(r[60]), "r"(r[61]), "r"(r[62]), "r"(r[63])
                 : "memory");
}

__device__ __forceinline__ void tm_st16(unsigned taddr, const unsigned (&r)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};\n"
                 :
                 : "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
                 : "memory");
}


// 32 complex values per thread at columns c .. c + 63 (value j: columns c + 2j, c + 2j + 1)
__device__ __forceinline__ void tm_load32c(unsigned taddr, float2 (&v)[32]) {
    unsigned r[64];
    tm_ld64(taddr, r);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
}
__device__ __forceinline__ void tm_store32c(unsigned taddr, const float2 (&v)[32]) {
    unsigned r[64];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        r[2 * j] = __float_as_uint(v[j].x);
        r[2 * j + 1] = __float_as_uint(v[j].y);
    }
    tm_st64(taddr, r);
}
// 8 complex values: columns c .. c + 15
__device__ __forceinline__ void tm_load8c(unsigned taddr, float2 (&v)[8]) {
    unsigned r[16];
    tm_ld16(taddr, r);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
}
__device__ __forceinline__ void tm_store8c(unsigned taddr, const float2 (&v)[8]) {
    unsigned r[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        r[2 * j] = __float_as_uint(v[j].x);
        r[2 * j + 1] = __float_as_uint(v[j].y);
    }
    tm_st16(taddr, r);
}

// 16 complex values from runtime columns: value j from columns a[j], a[j] + 1.
__device__ __forceinline__ void tm_ld2x16(const unsigned (&a)[16], unsigned (&r)[32]) {
    asm volatile(
        "{\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%32];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%2, %3}, [%33];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4, %5}, [%34];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%6, %7}, [%35];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8, %9}, [%36];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%10, %11}, [%37];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%12, %13}, [%38];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%14, %15}, [%39];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%16, %17}, [%40];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%18, %19}, [%41];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%20, %21}, [%42];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%22, %23}, [%43];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%24, %25}, [%44];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%26, %27}, [%45];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%28, %29}, [%46];\n"
        " tcgen05.ld.sync.aligned.32x32b.x2.b32 {%30, %31}, [%47];\n"
        " tcgen05.wait::ld.sync.aligned;\n}\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]), "r"(a[9]), "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]), "r"(a[15])
        : "memory");
}

// 16 complex values to runtime columns (value j to columns a[j], a[j] + 1).
__device__ __forceinline__ void tm_st2x16(const unsigned (&a)[16], const unsigned (&r)[32]) {
    asm volatile(
        "{\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%16, %17};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%1], {%18, %19};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%2], {%20, %21};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%3], {%22, %23};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%4], {%24, %25};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%5], {%26, %27};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%6], {%28, %29};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%7], {%30, %31};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%8], {%32, %33};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%9], {%34, %35};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%10], {%36, %37};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%11], {%38, %39};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%12], {%40, %41};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%13], {%42, %43};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%14], {%44, %45};\n"
        " tcgen05.st.sync.aligned.32x32b.x2.b32 [%15], {%46, %47};\n"
        "}\n"
        :
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]), "r"(a[9]), "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]), "r"(a[15]), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

// Rows (l + 32 q) of a 32-value column in tensor memory, q = (q0 + j) mod 32
// for j < 16: the 16 registers a term whose support lies in rows
// [32 q0, 32 q0 + 512) (mod 1024) needs, in that order.
__device__ __forceinline__ void tm_load16_rot(unsigned taddr, int q0, float2 (&v)[32]) {
    unsigned a[16], r[32];
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = taddr + 2u * (unsigned)((q0 + j) & 31);
    tm_ld2x16(a, r);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
}
__device__ __forceinline__ void tm_store16_rot(unsigned taddr, int q0, const float2 (&v)[32]) {
    unsigned a[16], r[32];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        a[j] = taddr + 2u * (unsigned)((q0 + j) & 31);
        r[2 * j] = __float_as_uint(v[j].x);
        r[2 * j + 1] = __float_as_uint(v[j].y);
    }
    tm_st2x16(a, r);
}

}  // namespace pce
