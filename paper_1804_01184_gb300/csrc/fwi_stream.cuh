// fwi_stream.cuh -- row-streaming time-step kernels (sm_103a).
//
// One CTA spans the whole computational row (4 consecutive columns per thread, float4
// loads and stores) and marches down a strip of TZ rows of one shot.  z-neighbours live in
// register queues (a ring of 2M rows, statically indexed inside a loop unrolled by 2M, so
// advancing it costs no moves); x-neighbours come from one shared-memory row (a ring of 2M
// rows for the p-like field, a double-buffered row for the v-like field).  One barrier per
// row.  The row lags the load front by 2M-1 rows:
//   front f     : p-like row f is loaded (register queue + shared ring)
//   f - M       : vz (half node f-M+1/2) from the register queue
//   j = f-2M+1  : vx row j from the shared ring, then p row j (D-x from the shared row,
//                 D-z from the vz queue)
// Every value outside the computational grid is zero (rows < 0 or >= Nz, columns >= Nx).
#pragma once
#include "fwi_kernels.cuh"
#include "fwi_tma.cuh"

namespace fwi {

constexpr int SHALO = 4;   // zero columns on each side of a shared row (one float4)

__device__ __forceinline__ float4 f4(float v) { return make_float4(v, v, v, v); }
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
template <int M>
__device__ __forceinline__ float4 row_dplus(const float *row, int c0, const Stencil &st)
{
    float w[12];
    const float4 a = ld4(row + c0 - 4), b = ld4(row + c0), c = ld4(row + c0 + 4);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    w[8] = c.x; w[9] = c.y; w[10] = c.z; w[11] = c.w;
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float g = 0.f;
#pragma unroll
        for (int k = 1; k <= M; ++k) g = fmaf(st.c[k - 1], w[4 + q + k] - w[4 + q - k + 1], g);
        o[q] = g;
    }
    return make_float4(o[0], o[1], o[2], o[3]);
}

// D- along x of a shared half-node row at the four nodes c0 .. c0+3:
// sum_k c_k (g[i+k-1] - g[i-k]) needs columns c0-4 .. c0+6.
template <int M>
__device__ __forceinline__ float4 row_dminus(const float *row, int c0, const Stencil &st)
{
    float w[12];
    const float4 a = ld4(row + c0 - 4), b = ld4(row + c0), c = ld4(row + c0 + 4);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    w[8] = c.x; w[9] = c.y; w[10] = c.z; w[11] = c.w;
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float g = 0.f;
#pragma unroll
        for (int k = 1; k <= M; ++k) g = fmaf(st.c[k - 1], w[4 + q + k - 1] - w[4 + q - k], g);
        o[q] = g;
    }
    return make_float4(o[0], o[1], o[2], o[3]);
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

// ------------------------------------------------------------------ forward step (S3)
//
// Same arithmetic as the staggered step: v^{n+1/2} = d_v (v^{n-1/2} - dt b D+ p^n),
// p^{n+1} = d_p (p^n - dt K D-.v^{n+1/2}) + dt K w_n beta / dx^2.
// grid = (ceil(Nz / tz), shots), block = NT threads with 4 * NT >= Nx; tz multiple of 2M.
// Global values one forward iteration (front f) consumes, loaded one iteration ahead.
struct FwdRow {
    float4 p, vz, bz, vx, bx, K;
    float azh, az;
};

template <int M>
__device__ __forceinline__ FwdRow fwd_load(int f, bool act, int c0, const Dims &d, const float *P0, const float *VZ0,
                                           const float *VX0, const Model &mo)
{
    FwdRow w;
    w.p = w.vz = w.bz = w.vx = w.bx = w.K = f4(0.f);
    w.azh = w.az = 0.f;
    const int r = f - M, j = f - 2 * M + 1;
    if (act && f >= 0 && f < d.Nz) w.p = ldg4(P0 + f * d.Px + c0);
    if (act && r >= 0 && r < d.Nz) {
        const int o = r * d.Px + c0;
        w.vz = ldg4(VZ0 + o);
        w.bz = ldg4(mo.bz + o);
        w.azh = __ldg(mo.azh + r);
    }
    if (act && j >= 0 && j < d.Nz) {
        const int o = j * d.Px + c0;
        w.vx = ldg4(VX0 + o);
        w.bx = ldg4(mo.bx + o);
        w.K = ldg4(mo.K + o);
        w.az = __ldg(mo.az + j);
    }
    return w;
}

template <int M>
__global__ void __launch_bounds__(384) k_fwd_stream(const float *__restrict__ p0, const float *__restrict__ vx0,
                                                   const float *__restrict__ vz0, float *__restrict__ p1,
                                                   float *__restrict__ vx1, float *__restrict__ vz1, Model mo,
                                                   Dims d, Stencil st, Source src, int n, int tz)
{
    constexpr int R = 2 * M;
    extern __shared__ __align__(128) float sm[];
    const int NT = blockDim.x, L = row_len(NT);
    float *ring = sm;                 // R rows of p^n
    float *vxb = sm + R * L;          // 2 rows of vx^{n+1/2}
    const int t = threadIdx.x, c0 = 4 * t;
    const bool act = c0 < d.Nx;
    for (int k = t; k < (R + 2) * L; k += NT) sm[k] = 0.f;
    const int z0 = blockIdx.x * tz, s = blockIdx.y;
    const long long so = (long long)s * d.Np;
    const float *P0 = p0 + so, *VX0 = vx0 + so, *VZ0 = vz0 + so;
    float *P1 = p1 + so, *VX1 = vx1 + so, *VZ1 = vz1 + so;
    const SrcCells sc = src_cells(src, s, d.Px);
    const float wn = __ldg(src.wav + n);
    float4 axv = f4(0.f), axhv = f4(0.f);
    if (act) { axv = ldg4(mo.ax + c0); axhv = ldg4(mo.axh + c0); }
    float4 pq[R], vq[R];
#pragma unroll
    for (int k = 0; k < R; ++k) { pq[k] = f4(0.f); vq[k] = f4(0.f); }
    const int zend = min(z0 + tz, d.Nz);
    FwdRow nxt = fwd_load<M>(z0 - R, act, c0, d, P0, VZ0, VX0, mo);
    __syncthreads();
    for (int fb = z0 - R; fb < zend + R; fb += R) {
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int f = fb + u;
            const FwdRow cur = nxt;
            nxt = fwd_load<M>(f + 1, act, c0, d, P0, VZ0, VX0, mo);
            // 1. p^n row f
            pq[u] = cur.p;
            st4(ring + u * L + SHALO + c0, cur.p);
            // 2. vz at half node r + 1/2, r = f - M: D+z from rows f-2M+1 .. f
            const int r = f - M;
            float4 vz = f4(0.f);
            if (act && r >= 0 && r < d.Nz) {
                float4 g = f4(0.f);
#pragma unroll
                for (int k = 1; k <= M; ++k)
                    g = fma4(st.c[k - 1], pq[(u - M + k + 2 * R) % R] - pq[(u - M - k + 1 + 2 * R) % R], g);
                vz = mask4((cur.azh * axv) * (cur.vz - cur.bz * g), c0, d.Nx);
                if (r >= z0 && r < zend) st4(VZ1 + r * d.Px + c0, vz);
            }
            vq[u] = vz;
            // 3. vx and p at row j = f - 2M + 1
            const int j = f - R + 1;
            const bool row = j >= z0 && j < zend;     // CTA-uniform
            float4 vx = f4(0.f);
            if (row && act) {
                const float4 g = row_dplus<M>(ring + ((u + 1) % R) * L + SHALO, c0, st);
                vx = mask4((cur.az * axhv) * (cur.vx - cur.bx * g), c0, d.Nx);
                st4(VX1 + j * d.Px + c0, vx);
            }
            float *vrow = vxb + (u & 1) * L + SHALO;
            if (row) st4(vrow + c0, vx);
            __syncthreads();
            if (row && act) {
                float4 dv = row_dminus<M>(vrow, c0, st);
#pragma unroll
                for (int k = 1; k <= M; ++k)
                    dv = fma4(st.c[k - 1], vq[(u - M + k + 2 * R) % R] - vq[(u + 1 - k - M + 2 * R) % R], dv);
                float4 pn = (cur.az * axv) * (pq[(u + 1) % R] - cur.K * dv);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (sc.j[k] == j && sc.i[k] >= c0 && sc.i[k] < c0 + 4)
                        addc(pn, sc.i[k] - c0, comp(cur.K, sc.i[k] - c0) * wn * sc.w[k]);
                st4(P1 + j * d.Px + c0, mask4(pn, c0, d.Nx));
            }
        }
    }
}

// ------------------------------------------------------------- adjoint step (S7)
//
// Transpose of k_fwd_stream's step with the cross-correlation fused in (reverse step n):
//   q = d_p pbar^{n+1};  u = d_v (vbar + dt D+ (K q))  -> new vbar;  pbar^n = q + dt D- (b u)
//   accB += u dt D+ p^n  (g_b = -accB);  accK += pbar^{n+1} (p^{n+1} - d_p p^n)  (g_K = accK / K)
// Register queues (2M rows each): K q, p^n, bz uz.  Shared rings: K q, p^n; one bx ux row.
template <int M>
__global__ void __launch_bounds__(384) k_adj_stream(const float *__restrict__ ap0, const float *__restrict__ avx0,
                                                   const float *__restrict__ avz0, float *__restrict__ ap1,
                                                   float *__restrict__ avx1, float *__restrict__ avz1, Model mo,
                                                   const float *__restrict__ pn, const float *__restrict__ pn1,
                                                   float *__restrict__ accK, float *__restrict__ accBx,
                                                   float *__restrict__ accBz, Dims d, Stencil st, int tz)
{
    constexpr int R = 2 * M;
    extern __shared__ __align__(128) float sm[];
    const int NT = blockDim.x, L = row_len(NT);
    float *qring = sm;                // R rows of K d_p pbar^{n+1}
    float *pring = sm + R * L;        // R rows of p^n
    float *bub = sm + 2 * R * L;      // 2 rows of bx ux
    const int t = threadIdx.x, c0 = 4 * t;
    const bool act = c0 < d.Nx;
    for (int k = t; k < (2 * R + 2) * L; k += NT) sm[k] = 0.f;
    const int z0 = blockIdx.x * tz, s = blockIdx.y;
    const long long so = (long long)s * d.Np;
    const float *A0 = ap0 + so, *AX0 = avx0 + so, *AZ0 = avz0 + so, *PN = pn + so, *PN1 = pn1 + so;
    float *A1 = ap1 + so, *AX1 = avx1 + so, *AZ1 = avz1 + so;
    float *GK = accK + so, *GX = accBx + so, *GZ = accBz + so;
    float4 axv = f4(0.f), axhv = f4(0.f);
    if (act) { axv = ldg4(mo.ax + c0); axhv = ldg4(mo.axh + c0); }
    float4 qq[R], pq[R], bq[R];
#pragma unroll
    for (int k = 0; k < R; ++k) { qq[k] = f4(0.f); pq[k] = f4(0.f); bq[k] = f4(0.f); }
    __syncthreads();
    const int zend = min(z0 + tz, d.Nz);
    for (int fb = z0 - R; fb < zend + R; fb += R) {
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int f = fb + u;
            float4 qf = f4(0.f), pf = f4(0.f);
            if (act && f >= 0 && f < d.Nz) {
                const int o = f * d.Px + c0;
                qf = (__ldg(mo.az + f) * axv) * ldg4(mo.K + o) * ldg4(A0 + o);
                pf = ldg4(PN + o);
            }
            qq[u] = qf;
            pq[u] = pf;
            st4(qring + u * L + SHALO + c0, qf);
            st4(pring + u * L + SHALO + c0, pf);
            // uz at half node r + 1/2, r = f - M
            const int r = f - M;
            float4 bu = f4(0.f);
            if (act && r >= 0 && r < d.Nz) {
                float4 gq = f4(0.f), gp = f4(0.f);
#pragma unroll
                for (int k = 1; k <= M; ++k) {
                    const int a = (u - M + k + 2 * R) % R, b = (u - M - k + 1 + 2 * R) % R;
                    gq = fma4(st.c[k - 1], qq[a] - qq[b], gq);
                    gp = fma4(st.c[k - 1], pq[a] - pq[b], gp);
                }
                const int o = r * d.Px + c0;
                float4 uz = (__ldg(mo.azh + r) * axv) * (ldg4(AZ0 + o) + gq);
                uz = mask4(uz, c0, d.Nx);
                bu = ldg4(mo.bz + o) * uz;
                if (r >= z0 && r < zend) {
                    st4(AZ1 + o, uz);
                    st4(GZ + o, ldg4(GZ + o) + uz * gp);
                }
            }
            bq[u] = bu;
            // ux and pbar^n at row j = f - 2M + 1
            const int j = f - R + 1;
            const bool row = j >= z0 && j < zend;
            float4 bux = f4(0.f);
            if (row && act) {
                const int o = j * d.Px + c0;
                const int slot = (u + 1) % R;
                const float4 gq = row_dplus<M>(qring + slot * L + SHALO, c0, st);
                const float4 gp = row_dplus<M>(pring + slot * L + SHALO, c0, st);
                float4 ux = (__ldg(mo.az + j) * axhv) * (ldg4(AX0 + o) + gq);
                ux = mask4(ux, c0, d.Nx);
                st4(AX1 + o, ux);
                st4(GX + o, ldg4(GX + o) + ux * gp);
                bux = ldg4(mo.bx + o) * ux;
            }
            float *brow = bub + (u & 1) * L + SHALO;
            if (row) st4(brow + c0, bux);
            __syncthreads();
            if (row && act) {
                const int o = j * d.Px + c0;
                float4 dv = row_dminus<M>(brow, c0, st);
#pragma unroll
                for (int k = 1; k <= M; ++k)
                    dv = fma4(st.c[k - 1], bq[(u - M + k + 2 * R) % R] - bq[(u + 1 - k - M + 2 * R) % R], dv);
                const float4 dp = __ldg(mo.az + j) * axv;
                const float4 a = ldg4(A0 + o);
                st4(A1 + o, mask4(dp * a + dv, c0, d.Nx));
                st4(GK + o, ldg4(GK + o) + a * (ldg4(PN1 + o) - dp * pq[(u + 1) % R]));
            }
        }
    }
}

// ------------------------------------------------------------------------ Born (S6)
//
// Background (p, v) and scattered (q, u) fields stepped together:
//   u^{n+1/2} = d_v (u^{n-1/2} - dt b D+ q^n - dt db D+ p^n)
//   q^{n+1}   = d_p (q^n - dt K D-.u^{n+1/2} - dt dK D-.v^{n+1/2}) + dt dK w_n beta / dx^2
template <int M>
__global__ void __launch_bounds__(384) k_born_stream(const float *__restrict__ p0, const float *__restrict__ vx0,
                                                    const float *__restrict__ vz0, const float *__restrict__ q0,
                                                    const float *__restrict__ ux0, const float *__restrict__ uz0,
                                                    float *__restrict__ p1, float *__restrict__ vx1,
                                                    float *__restrict__ vz1, float *__restrict__ q1,
                                                    float *__restrict__ ux1, float *__restrict__ uz1, Model mo,
                                                    Pert pe, Dims d, Stencil st, Source src, int n, int tz)
{
    constexpr int R = 2 * M;
    extern __shared__ __align__(128) float sm[];
    const int NT = blockDim.x, L = row_len(NT);
    float *pring = sm, *qring = sm + R * L;     // R rows each of p^n, q^n
    float *vb = sm + 2 * R * L;                 // 2 rows of vx^{n+1/2}
    float *ub = sm + (2 * R + 2) * L;           // 2 rows of ux^{n+1/2}
    const int t = threadIdx.x, c0 = 4 * t;
    const bool act = c0 < d.Nx;
    for (int k = t; k < (2 * R + 4) * L; k += NT) sm[k] = 0.f;
    const int z0 = blockIdx.x * tz, s = blockIdx.y;
    const long long so = (long long)s * d.Np;
    const float *P0 = p0 + so, *VX0 = vx0 + so, *VZ0 = vz0 + so, *Q0 = q0 + so, *UX0 = ux0 + so, *UZ0 = uz0 + so;
    float *P1 = p1 + so, *VX1 = vx1 + so, *VZ1 = vz1 + so, *Q1 = q1 + so, *UX1 = ux1 + so, *UZ1 = uz1 + so;
    const SrcCells sc = src_cells(src, s, d.Px);
    const float wn = __ldg(src.wav + n);
    float4 axv = f4(0.f), axhv = f4(0.f);
    if (act) { axv = ldg4(mo.ax + c0); axhv = ldg4(mo.axh + c0); }
    float4 vq[R], uq[R];      // vz, uz queues; p and q z-neighbours are read from the shared rings
#pragma unroll
    for (int k = 0; k < R; ++k) { vq[k] = f4(0.f); uq[k] = f4(0.f); }
    __syncthreads();
    const int zend = min(z0 + tz, d.Nz);
    for (int fb = z0 - R; fb < zend + R; fb += R) {
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int f = fb + u;
            float4 pf = f4(0.f), qf = f4(0.f);
            if (act && f >= 0 && f < d.Nz) { pf = ldg4(P0 + f * d.Px + c0); qf = ldg4(Q0 + f * d.Px + c0); }
            st4(pring + u * L + SHALO + c0, pf);
            st4(qring + u * L + SHALO + c0, qf);
            const int r = f - M;
            float4 vz = f4(0.f), uz = f4(0.f);
            if (act && r >= 0 && r < d.Nz) {
                float4 gp = f4(0.f), gq = f4(0.f);
#pragma unroll
                for (int k = 1; k <= M; ++k) {
                    const int a = (u - M + k + 2 * R) % R, b = (u - M - k + 1 + 2 * R) % R;
                    gp = fma4(st.c[k - 1], ld4(pring + a * L + SHALO + c0) - ld4(pring + b * L + SHALO + c0), gp);
                    gq = fma4(st.c[k - 1], ld4(qring + a * L + SHALO + c0) - ld4(qring + b * L + SHALO + c0), gq);
                }
                const int o = r * d.Px + c0;
                const float4 fz = __ldg(mo.azh + r) * axv, b = ldg4(mo.bz + o);
                vz = mask4(fz * (ldg4(VZ0 + o) - b * gp), c0, d.Nx);
                uz = mask4(fz * (ldg4(UZ0 + o) - b * gq - ldg4(pe.dbz + o) * gp), c0, d.Nx);
                if (r >= z0 && r < zend) { st4(VZ1 + o, vz); st4(UZ1 + o, uz); }
            }
            vq[u] = vz;
            uq[u] = uz;
            const int j = f - R + 1;
            const bool row = j >= z0 && j < zend;
            float4 vx = f4(0.f), ux = f4(0.f);
            if (row && act) {
                const int o = j * d.Px + c0;
                const int slot = (u + 1) % R;
                const float4 gp = row_dplus<M>(pring + slot * L + SHALO, c0, st);
                const float4 gq = row_dplus<M>(qring + slot * L + SHALO, c0, st);
                const float4 fx = __ldg(mo.az + j) * axhv, b = ldg4(mo.bx + o);
                vx = mask4(fx * (ldg4(VX0 + o) - b * gp), c0, d.Nx);
                ux = mask4(fx * (ldg4(UX0 + o) - b * gq - ldg4(pe.dbx + o) * gp), c0, d.Nx);
                st4(VX1 + o, vx);
                st4(UX1 + o, ux);
            }
            float *vrow = vb + (u & 1) * L + SHALO, *urow = ub + (u & 1) * L + SHALO;
            if (row) { st4(vrow + c0, vx); st4(urow + c0, ux); }
            __syncthreads();
            if (row && act) {
                const int o = j * d.Px + c0;
                float4 dv = row_dminus<M>(vrow, c0, st), du = row_dminus<M>(urow, c0, st);
#pragma unroll
                for (int k = 1; k <= M; ++k) {
                    const int a = (u - M + k + 2 * R) % R, b = (u + 1 - k - M + 2 * R) % R;
                    dv = fma4(st.c[k - 1], vq[a] - vq[b], dv);
                    du = fma4(st.c[k - 1], uq[a] - uq[b], du);
                }
                const float4 K = ldg4(mo.K + o), dK = ldg4(pe.dK + o), fp = __ldg(mo.az + j) * axv;
                const int slot = (u + 1) % R;
                float4 pn = fp * (ld4(pring + slot * L + SHALO + c0) - K * dv);
                float4 qn = fp * (ld4(qring + slot * L + SHALO + c0) - K * du - dK * dv);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (sc.j[k] == j && sc.i[k] >= c0 && sc.i[k] < c0 + 4) {
                        const int q = sc.i[k] - c0;
                        addc(pn, q, comp(K, q) * wn * sc.w[k]);
                        addc(qn, q, comp(dK, q) * wn * sc.w[k]);
                    }
                st4(P1 + o, mask4(pn, c0, d.Nx));
                st4(Q1 + o, mask4(qn, c0, d.Nx));
            }
        }
    }
}

// ------------------------------------------------- forward step, TMA-fed (S3)
//
// The row-streaming forward step with every global input row brought into shared memory by
// the TMA engine PD rows ahead of use: p^n (ring of 2M + PD rows: the register queue and the
// D+x stencil read it), vz^{n-1/2} and bz (consumed at lag M), vx^{n-1/2}, bx, K (lag 2M-1)
// in rings of PD + 1 rows.  Stage g (front f = f0 + g) carries p row f, vz/bz row f - M and
// vx/bx/K row f - 2M + 1 on one mbarrier.
constexpr int PD = 4;   // prefetch distance in rows

template <int M>
__global__ void __launch_bounds__(384, 1) k_fwd_tma(const float *__restrict__ p0, const float *__restrict__ vx0,
                                                   const float *__restrict__ vz0, float *__restrict__ p1,
                                                   float *__restrict__ vx1, float *__restrict__ vz1, Model mo,
                                                   Dims d, Stencil st, Source src, int n, int tz, int *status)
{
    constexpr int R = 2 * M, SP = R + PD, S = PD + 1;
    extern __shared__ __align__(128) float sm[];
    __shared__ int abort_flag;
    const int NT = blockDim.x, L = row_len(NT);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);   // S mbarriers (first 64 bytes)
    float *pr = sm + 16;
    float *vzr = pr + SP * L, *bzr = vzr + S * L, *vxr = bzr + S * L, *bxr = vxr + S * L, *Kr = bxr + S * L;
    float *vxb = Kr + S * L;
    const int t = threadIdx.x, c0 = 4 * t;
    const bool act = c0 < d.Nx;     // computes
    const bool wr = c0 < d.Px;      // writes (zeros beyond Nx): every written row is fully defined,
                                    // so whole-row TMA loads never see stale padding
    for (int k = 16 + t; k < 16 + (SP + 5 * S + 2) * L; k += NT) sm[k] = 0.f;
    fence_async_shared();
    if (t == 0) {
        for (int k = 0; k < S; ++k) mbar_init(bar + k, 1);
        mbar_init_fence();
        abort_flag = 0;
    }
    const int z0 = blockIdx.x * tz, s = blockIdx.y;
    const long long so = (long long)s * d.Np;
    const float *P0 = p0 + so, *VX0 = vx0 + so, *VZ0 = vz0 + so;
    float *P1 = p1 + so, *VX1 = vx1 + so, *VZ1 = vz1 + so;
    const SrcCells sc = src_cells(src, s, d.Px);
    const float wn = __ldg(src.wav + n);
    float4 axv = f4(0.f), axhv = f4(0.f);
    if (act) { axv = ldg4(mo.ax + c0); axhv = ldg4(mo.axh + c0); }
    float4 pq[R], vq[R];
#pragma unroll
    for (int k = 0; k < R; ++k) { pq[k] = f4(0.f); vq[k] = f4(0.f); }
    const int zend = min(z0 + tz, d.Nz);
    const int f0 = z0 - R;
    const int nit = ((zend + R - f0 + R - 1) / R) * R;   // iterations of the unrolled loop
    const uint32_t rowb = (uint32_t)d.Px * 4u;
    // producer: stage g -> rings (one elected thread)
    auto issue = [&](int g) {
        const int f = f0 + g, r = f - M, j = f - R + 1;
        const bool vf = f >= 0 && f < d.Nz, vr = r >= 0 && r < d.Nz, vj = j >= 0 && j < d.Nz;
        uint64_t *b = bar + g % S;
        mbar_arrive_expect_tx(b, rowb * ((vf ? 1u : 0u) + (vr ? 2u : 0u) + (vj ? 3u : 0u)));
        const int sp = g % SP, so1 = g % S;
        if (vf) tma_load_1d(pr + sp * L + SHALO, P0 + (long long)f * d.Px, rowb, b);
        if (vr) {
            tma_load_1d(vzr + so1 * L + SHALO, VZ0 + (long long)r * d.Px, rowb, b);
            tma_load_1d(bzr + so1 * L + SHALO, mo.bz + (long long)r * d.Px, rowb, b);
        }
        if (vj) {
            tma_load_1d(vxr + so1 * L + SHALO, VX0 + (long long)j * d.Px, rowb, b);
            tma_load_1d(bxr + so1 * L + SHALO, mo.bx + (long long)j * d.Px, rowb, b);
            tma_load_1d(Kr + so1 * L + SHALO, mo.K + (long long)j * d.Px, rowb, b);
        }
    };
    __syncthreads();
    if (t == 0)
        for (int g = 0; g < PD && g < nit; ++g) issue(g);
    for (int fb = f0; fb < f0 + nit; fb += R) {
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int f = fb + u, g = f - f0;
            if (!mbar_wait(bar + g % S, (uint32_t)((g / S) & 1))) {
                atomicOr(status, ST_ETIMEOUT);
                abort_flag = 1;
            }
            const int sp = g % SP, so1 = g % S;
            // 1. p^n row f into the register queue
            pq[u] = (act && f >= 0 && f < d.Nz) ? ld4(pr + sp * L + SHALO + c0) : f4(0.f);
            // 2. vz at half node r + 1/2, r = f - M
            const int r = f - M;
            float4 vz = f4(0.f);
            if (act && r >= 0 && r < d.Nz) {
                float4 gz = f4(0.f);
#pragma unroll
                for (int k = 1; k <= M; ++k)
                    gz = fma4(st.c[k - 1], pq[(u - M + k + 2 * R) % R] - pq[(u - M - k + 1 + 2 * R) % R], gz);
                vz = mask4((__ldg(mo.azh + r) * axv) *
                               (ld4(vzr + so1 * L + SHALO + c0) - ld4(bzr + so1 * L + SHALO + c0) * gz), c0, d.Nx);
            }
            if (wr && r >= z0 && r < zend) st4(VZ1 + r * d.Px + c0, vz);
            vq[u] = vz;
            // 3. vx and p at row j = f - 2M + 1
            const int j = f - R + 1;
            const bool row = j >= z0 && j < zend;
            float4 vx = f4(0.f), Kv = f4(0.f);
            if (row && act) {
                const float4 gx = row_dplus<M>(pr + ((g - R + 1 + SP) % SP) * L + SHALO, c0, st);
                vx = mask4((__ldg(mo.az + j) * axhv) *
                               (ld4(vxr + so1 * L + SHALO + c0) - ld4(bxr + so1 * L + SHALO + c0) * gx), c0, d.Nx);
                Kv = ld4(Kr + so1 * L + SHALO + c0);
            }
            if (row && wr) st4(VX1 + j * d.Px + c0, vx);
            float *vrow = vxb + (u & 1) * L + SHALO;
            if (row) st4(vrow + c0, vx);
            __syncthreads();
            if (abort_flag) {   // drain the stages still in flight (bounded), then leave
                if (t == 0)
                    for (int h = g + 1; h < g + PD && h < nit; ++h) mbar_wait(bar + h % S, (uint32_t)((h / S) & 1));
                return;
            }
            if (t == 0 && g + PD < nit) {
                fence_async_shared();
                issue(g + PD);
            }
            if (row && wr) {
                float4 pn = f4(0.f);
                if (act) {
                    float4 dv = row_dminus<M>(vrow, c0, st);
#pragma unroll
                    for (int k = 1; k <= M; ++k)
                        dv = fma4(st.c[k - 1], vq[(u - M + k + 2 * R) % R] - vq[(u + 1 - k - M + 2 * R) % R], dv);
                    pn = (__ldg(mo.az + j) * axv) * (pq[(u + 1) % R] - Kv * dv);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (sc.j[k] == j && sc.i[k] >= c0 && sc.i[k] < c0 + 4)
                            addc(pn, sc.i[k] - c0, comp(Kv, sc.i[k] - c0) * wn * sc.w[k]);
                    pn = mask4(pn, c0, d.Nx);
                }
                st4(P1 + j * d.Px + c0, pn);
            }
        }
    }
}

}  // namespace fwi
