// fwi_stream.cuh -- float4 helpers and row stencils shared by the streaming time-step kernels.
//
// A streaming kernel marches down rows; 4 consecutive columns live in one float4.  The
// row stencils below evaluate the staggered x-derivatives of four outputs from a row staged in
// shared memory with a 4-column zero halo (SHALO) on each side.
#pragma once
#include "fwi_kernels.cuh"

namespace fwi {

constexpr int SHALO = 4;   // zero columns on each side of a shared row (one float4)

// shared-memory address of a generic pointer into shared memory (for cp.async)
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float4 f4(float v) { return make_float4(v, v, v, v); }

// Packed FP32x2 arithmetic (sm_100+): two lanes of a float4 per instruction, each component
// rounded exactly as the scalar operation.
__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cat4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
// a * b + c
__device__ __forceinline__ float4 pfma(const float4 &a, const float4 &b, const float4 &c)
{
    return cat4(__ffma2_rn(lo2(a), lo2(b), lo2(c)), __ffma2_rn(hi2(a), hi2(b), hi2(c)));
}
// s * b + c
__device__ __forceinline__ float4 pfma(float s, const float4 &b, const float4 &c)
{
    const float2 s2 = make_float2(s, s);
    return cat4(__ffma2_rn(s2, lo2(b), lo2(c)), __ffma2_rn(s2, hi2(b), hi2(c)));
}
__device__ __forceinline__ float4 pmul(const float4 &a, const float4 &b)
{
    return cat4(__fmul2_rn(lo2(a), lo2(b)), __fmul2_rn(hi2(a), hi2(b)));
}
__device__ __forceinline__ float4 pmul(float s, const float4 &b)
{
    const float2 s2 = make_float2(s, s);
    return cat4(__fmul2_rn(s2, lo2(b)), __fmul2_rn(s2, hi2(b)));
}
__device__ __forceinline__ float4 padd(const float4 &a, const float4 &b)
{
    return cat4(__fadd2_rn(lo2(a), lo2(b)), __fadd2_rn(hi2(a), hi2(b)));
}
// a - b (b * -1 + a: exact product, one rounding)
__device__ __forceinline__ float4 psub(const float4 &a, const float4 &b)
{
    const float2 m = make_float2(-1.f, -1.f);
    return cat4(__ffma2_rn(lo2(b), m, lo2(a)), __ffma2_rn(hi2(b), m, hi2(a)));
}
// c + s * (a - b): one stencil tap on a float4
__device__ __forceinline__ float4 ptap(float s, const float4 &a, const float4 &b, const float4 &c)
{
    return pfma(s, psub(a, b), c);
}
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float4 operator+(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 operator-(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ __forceinline__ float4 operator*(float4 a, float4 b) { return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w); }
__device__ __forceinline__ float4 operator*(float s, float4 b) { return make_float4(s * b.x, s * b.y, s * b.z, s * b.w); }
__device__ __forceinline__ float4 fma4(float s, float4 a, float4 c) { return make_float4(fmaf(s, a.x, c.x), fmaf(s, a.y, c.y), fmaf(s, a.z, c.z), fmaf(s, a.w, c.w)); }
__device__ __forceinline__ float comp(const float4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
__device__ __forceinline__ void addc(float4 &v, int k, float a)
{
    if (k == 0) v.x += a; else if (k == 1) v.y += a; else if (k == 2) v.z += a; else v.w += a;
}
// zero the components at columns >= Nx (c0 = first column of the float4)
__device__ __forceinline__ float4 mask4(float4 v, int c0, int Nx)
{
    if (c0 + 3 >= Nx) {
        if (c0 + 1 >= Nx) v.y = 0.f;
        if (c0 + 2 >= Nx) v.z = 0.f;
        if (c0 + 3 >= Nx) v.w = 0.f;
        if (c0 >= Nx) v.x = 0.f;
    }
    return v;
}

// D+ along x of a shared row at the four half nodes c0+1/2 .. c0+3+1/2 (c0 = 4*tid):
// sum_k c_k (f[i+k] - f[i-k+1]) needs columns c0-3 .. c0+7 = three aligned float4.
// b: the row's float4 at c0 when the caller already holds it in registers (one shared load
// fewer), else read here.
template <int M>
__device__ __forceinline__ float4 row_dplus(const float *row, int c0, const float4 &b, const float *cf)
{
    float w[12];
    const float4 a = ld4(row + c0 - 4), c = ld4(row + c0 + 4);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    w[8] = c.x; w[9] = c.y; w[10] = c.z; w[11] = c.w;
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float g = 0.f;
#pragma unroll
        for (int k = 1; k <= M; ++k) g = fmaf(cf[k - 1], w[4 + q + k] - w[4 + q - k + 1], g);
        o[q] = g;
    }
    return make_float4(o[0], o[1], o[2], o[3]);
}

template <int M>
__device__ __forceinline__ float4 row_dplus(const float *row, int c0, const float *cf)
{
    return row_dplus<M>(row, c0, ld4(row + c0), cf);
}

// D- along x of a shared half-node row at the four nodes c0 .. c0+3:
// sum_k c_k (g[i+k-1] - g[i-k]) needs columns c0-4 .. c0+6.
template <int M>
__device__ __forceinline__ float4 row_dminus(const float *row, int c0, const float4 &b, const float *cf)
{
    float w[12];
    const float4 a = ld4(row + c0 - 4), c = ld4(row + c0 + 4);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    w[8] = c.x; w[9] = c.y; w[10] = c.z; w[11] = c.w;
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float g = 0.f;
#pragma unroll
        for (int k = 1; k <= M; ++k) g = fmaf(cf[k - 1], w[4 + q + k - 1] - w[4 + q - k], g);
        o[q] = g;
    }
    return make_float4(o[0], o[1], o[2], o[3]);
}

template <int M>
__device__ __forceinline__ float4 row_dminus(const float *row, int c0, const float *cf)
{
    return row_dminus<M>(row, c0, ld4(row + c0), cf);
}

// Shared layout of one row: SHALO zeros, 4*NT columns, SHALO zeros.
__device__ __forceinline__ int row_len(int nthreads) { return 4 * nthreads + 2 * SHALO; }

// Per-shot source footprint decoded to (row, column) once per CTA.
struct SrcCells {
    int j[4], i[4];
    float w[4];
};
__device__ __forceinline__ SrcCells src_cells(const Source &src, int s, int Px)
{
    SrcCells c;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const long long o = src.idx[4 * s + k];
        c.j[k] = (int)(o / Px);
        c.i[k] = (int)(o - (long long)c.j[k] * Px);
        c.w[k] = src.w[4 * s + k];
    }
    return c;
}

}  // namespace fwi
