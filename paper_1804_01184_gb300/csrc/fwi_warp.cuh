// fwi_warp.cuh -- warp-strip streaming time-step kernels (sm_103a).
//
// Every warp owns a strip of 128 columns (4 per lane, float4 accesses) and tz rows of one
// shot, and marches down it independently: z-neighbours in register queues (a ring of 2M
// rows indexed statically inside a loop unrolled by 2M), x-neighbours in a per-warp
// shared row with an 8-column halo, one __syncwarp per row and no block barriers.  Lanes 0
// and 31 also stage the x-halo of p and compute the v_x halo columns the divergence of the
// strip's edge columns needs.  Global loads of row f+1 are issued before row f is computed.
// Every value outside the computational grid is zero; every lane whose float4 starts below
// the row pitch writes it (zeros beyond Nx), so written rows are fully defined.
#pragma once
#include "fwi_stream.cuh"

namespace fwi {

constexpr int WS = 128;             // strip width (columns)
constexpr int WH = 8;               // shared-row halo (columns each side)
constexpr int WROW = WS + 2 * WH;   // shared row length (floats)

struct Strip {
    int x0, z0, s;      // strip origin and shot
};

// warp -> strip: blockIdx.x * warps_per_block + warp, laid out as (x-strip, z-strip, shot)
__device__ __forceinline__ Strip strip_of(const Dims &d, int tz, int nshots, bool &valid)
{
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nxs = (d.Nx + WS - 1) / WS, nzs = (d.Nz + tz - 1) / tz;
    valid = w < nxs * nzs * nshots;
    // the shot varies fastest: warps running together stream the same model rows (shared by
    // every shot of the launch) and find them in L1/L2
    Strip st;
    st.s = w % nshots;
    st.x0 = ((w / nshots) % nxs) * WS;
    st.z0 = (w / (nshots * nxs)) * tz;
    return st;
}

// float4 of field f at (row, column c), zero outside the grid (c multiple of 4)
__device__ __forceinline__ float4 ld_row4(const float *f, const Dims &d, int row, int c)
{
    if (row < 0 || row >= d.Nz || c < 0 || c >= d.Nx) return f4(0.f);
    return mask4(ldg4(f + row * d.Px + c), c, d.Nx);
}

// 16-byte asynchronous global -> shared copy (zero-filled when !valid), and its groups
__device__ __forceinline__ void cp16(void *dst, const void *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int WPD = 2;   // rows prefetched ahead by each warp

// copy one float4 of row `row`, column c of field f into shared dst (zeros outside the grid)
__device__ __forceinline__ void cp_row4(float *dst, const float *f, const Dims &d, int row, int c)
{
    const bool v = row >= 0 && row < d.Nz && c >= 0 && c < d.Nx;
    cp16(dst, v ? f + row * d.Px + c : f, v);
}

// Ring and stage depths are powers of two (slot = index & (depth - 1)); the depths exceed what
// the pipeline needs (p rows f-2M+1 .. f+WPD; WPD+1 stages).
constexpr int WRP = 16;   // p-like rings
constexpr int WNS = 4;    // staged rows
static_assert(WRP >= 2 * 4 + WPD && WNS >= WPD + 1, "ring too shallow");

// Does the strip hold any source cell of its shot? (uniform per warp)
__device__ __forceinline__ bool strip_has_src(const SrcCells &sc, int x0, int z0, int zend)
{
    bool h = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) h |= sc.i[k] >= x0 && sc.i[k] < x0 + WS && sc.j[k] >= z0 && sc.j[k] < zend;
    return h;
}

template <int M, int MINB>
__global__ void __launch_bounds__(64, MINB) k_fwd_warp(const float *__restrict__ p0, const float *__restrict__ vx0,
                                                      const float *__restrict__ vz0, float *__restrict__ p1,
                                                      float *__restrict__ vx1, float *__restrict__ vz1, Model mo,
                                                      Dims d, Stencil st, Source src, int n, int tz, int nshots)
{
    constexpr int R = 2 * M;
    __shared__ __align__(16) float sring[2][WRP][WROW];
    __shared__ __align__(16) float sstg[2][WNS][5][WROW];
    __shared__ __align__(16) float svx[2][2][WROW];
    bool valid;
    const Strip sp = strip_of(d, tz, nshots, valid);
    if (!valid) return;
    const int wid = (threadIdx.x >> 5) & 1, lane = threadIdx.x & 31;
    float(*ring)[WROW] = sring[wid];
    float(*stg)[5][WROW] = sstg[wid];
    float(*vxr)[WROW] = svx[wid];
    const int c0 = sp.x0 + 4 * lane;
    const int o0 = WH + 4 * lane;
    const bool edge = lane == 0 || lane == 31;
    const int hc = lane == 0 ? sp.x0 - 4 : sp.x0 + WS;    // v_x halo float4 column
    const int ho = lane == 0 ? WH - 4 : WH + WS;          // its shared offset
    const int hp = lane == 0 ? sp.x0 - 8 : sp.x0 + WS;    // first p halo float4 column
    const int hpo = lane == 0 ? 0 : WH + WS;              // its shared offset
    const bool wr = c0 < d.Px, act = c0 < d.Nx;
    const bool hv = edge && hc >= 0 && hc < d.Nx;          // halo v_x column inside the grid
    const bool hv0 = edge && hp >= 0 && hp < d.Nx, hv1 = edge && hp + 4 >= 0 && hp + 4 < d.Nx;
    for (int k = lane; k < 2 * WROW; k += 32) (&vxr[0][0])[k] = 0.f;
    const long long so = (long long)sp.s * d.Np;
    const float *P0 = p0 + so, *VX0 = vx0 + so, *VZ0 = vz0 + so;
    float *P1 = p1 + so, *VX1 = vx1 + so, *VZ1 = vz1 + so;
    const SrcCells sc = src_cells(src, sp.s, d.Px);
    const float wn = __ldg(src.wav + n);
    const float4 axv = act ? ldg4(mo.ax + c0) : f4(0.f), axhv = act ? ldg4(mo.axh + c0) : f4(0.f);
    const float4 axhh = hv ? ldg4(mo.axh + hc) : f4(0.f);
    const int z0 = sp.z0, zend = min(z0 + tz, d.Nz), f0 = z0 - R;
    const bool hsrc = strip_has_src(sc, sp.x0, z0, zend);
    // stage g: p row f0+g -> ring[g & (WRP-1)]; vz, bz row f0+g-M and vx, bx, K row f0+g-2M+1 -> stg[g & (WNS-1)]
    auto issue = [&](int g) {
        const int f = f0 + g, r = f - M, j = f - R + 1;
        const bool vf = f >= 0 && f < d.Nz, vr = r >= 0 && r < d.Nz, vj = j >= 0 && j < d.Nz;
        float *pr = ring[g & (WRP - 1)];
        float(*sg)[WROW] = stg[g & (WNS - 1)];
        const int of = f * d.Px, orr = r * d.Px, oj = j * d.Px;
        cp16(pr + o0, P0 + of + c0, vf && act);
        cp16(sg[0] + o0, VZ0 + orr + c0, vr && act);
        cp16(sg[1] + o0, mo.bz + orr + c0, vr && act);
        cp16(sg[2] + o0, VX0 + oj + c0, vj && act);
        cp16(sg[3] + o0, mo.bx + oj + c0, vj && act);
        cp16(sg[4] + o0, mo.K + oj + c0, vj && act);
        if (edge) {
            cp16(pr + hpo, P0 + of + hp, vf && hv0);
            cp16(pr + hpo + 4, P0 + of + hp + 4, vf && hv1);
            cp16(sg[2] + ho, VX0 + oj + hc, vj && hv);
            cp16(sg[3] + ho, mo.bx + oj + hc, vj && hv);
        }
        cp_commit();
    };
    float4 vq[R];   // vz rows r-2M+1 .. r (oldest first), shifted each row
#pragma unroll
    for (int k = 0; k < R; ++k) vq[k] = f4(0.f);
#pragma unroll
    for (int g = 0; g < WPD; ++g) issue(g);
    const int fend = zend + R - 1;
#pragma unroll 1
    for (int f = f0; f < fend; ++f) {
        {
            const int g = f - f0, u = f & 1;
            __syncwarp();                 // every lane is done with the slots issue() refills
            issue(g + WPD);
            cp_wait<WPD>();               // stage g has landed (for this lane)
            __syncwarp();                 // ... and for every lane
            float(*sg)[WROW] = stg[g & (WNS - 1)];
            // vz at half node r + 1/2, r = f - M: p rows r-M+1 .. r+M = stages g-2M+1 .. g
            const int r = f - M;
            float4 gz = f4(0.f);
#pragma unroll
            for (int k = 1; k <= M; ++k)
                gz = fma4(st.c[k - 1], ld4(ring[(g - M + k) & (WRP - 1)] + o0) - ld4(ring[(g - M - k + 1) & (WRP - 1)] + o0), gz);
            const float azh = (r >= 0 && r < d.Nz) ? __ldg(mo.azh + r) : 0.f;
            const float4 vz = mask4((azh * axv) * (ld4(sg[0] + o0) - ld4(sg[1] + o0) * gz), c0, d.Nx);
            if (wr && r >= z0 && r < zend) st4(VZ1 + r * d.Px + c0, vz);
#pragma unroll
            for (int q = 0; q < R - 1; ++q) vq[q] = vq[q + 1];
            vq[R - 1] = vz;
            // v_x at row j = f - 2M + 1 (own float4 and, on lanes 0/31, the halo float4)
            const int j = f - R + 1;
            const bool row = j >= z0 && j < zend;
            const float az = (j >= 0 && j < d.Nz) ? __ldg(mo.az + j) : 0.f;
            const float *prow = ring[(g - R + 1) & (WRP - 1)];
            const float4 vx = mask4((az * axhv) * (ld4(sg[2] + o0) - ld4(sg[3] + o0) * row_dplus<M>(prow, o0, st)), c0, d.Nx);
            float *vrow = vxr[u & 1];
            st4(vrow + o0, vx);
            if (edge) {
                const float4 vh = (az * axhh) * (ld4(sg[2] + ho) - ld4(sg[3] + ho) * row_dplus<M>(prow, ho, st));
                st4(vrow + ho, hv ? mask4(vh, hc, d.Nx) : f4(0.f));
            }
            if (row && wr) st4(VX1 + j * d.Px + c0, vx);
            __syncwarp();
            if (row && wr) {
                float4 dv = row_dminus<M>(vrow, o0, st);
#pragma unroll
                for (int k = 1; k <= M; ++k)   // vq[q] is vz row j - M + q
                    dv = fma4(st.c[k - 1], vq[M + k - 1] - vq[M - k], dv);
                const float4 Kv = ld4(sg[4] + o0);
                float4 pn = (az * axv) * (ld4(prow + o0) - Kv * dv);
                if (hsrc) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (sc.j[k] == j && sc.i[k] >= c0 && sc.i[k] < c0 + 4)
                            addc(pn, sc.i[k] - c0, comp(Kv, sc.i[k] - c0) * wn * sc.w[k]);
                }
                st4(P1 + j * d.Px + c0, mask4(pn, c0, d.Nx));
            }
        }
    }
    cp_wait<0>();
}

// fire-and-forget vector add into global memory (resolved in L2; one warp owns each address
// within a launch, so the order of additions is fixed)
__device__ __forceinline__ void red_add4(float *dst, float4 v)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// ------------------------------------------------------------- adjoint step (S7)
//
// Reverse step n, the transpose of k_fwd_warp's step, with the cross-correlation fused in:
//   q = K d_p pbar^{n+1};  u = d_v (vbar + dt D+ q) -> new vbar;  pbar^n = d_p pbar^{n+1} + dt D- (b u)
//   accBz/accBx += u dt D+ p^n    (g_b = -accB)
//   accK += p^n (pbar^n - d_p pbar^{n+1})      (g_K = accK / K)
// The last line pairs each pressure adjoint with its own snapshot one launch earlier than the
// textbook form sum pbar^{n+1} (p^{n+1} - d_p p^n); the receiver-cell remainder
// (R^T r_n) p^{n+1} is added by k_adj_inject_k.  Inputs are staged by cp.async WPD rows ahead.
template <int M, int MINB>
__global__ void __launch_bounds__(32, 2 * MINB) k_adj_warp(const float *__restrict__ ap0, const float *__restrict__ avx0,
                                                      const float *__restrict__ avz0, float *__restrict__ ap1,
                                                      float *__restrict__ avx1, float *__restrict__ avz1, Model mo,
                                                      const float *__restrict__ pn, float *__restrict__ accK,
                                                      float *__restrict__ accBx, float *__restrict__ accBz, Dims d,
                                                      Stencil st, int tz, int nshots)
{
    constexpr int R = 2 * M, NF = 7;
    // one warp per block
    __shared__ __align__(16) float spr[1][WRP][WROW];    // p^n rows (own + halo)
    __shared__ __align__(16) float sqr[1][R][WROW];      // K d_p pbar^{n+1} rows (own + halo)
    __shared__ __align__(16) float sstg[1][WNS][NF][WROW];
    __shared__ __align__(16) float sbu[1][2][WROW];      // bx ux rows (own + halo)
    bool valid;
    const Strip sp = strip_of(d, tz, nshots, valid);
    if (!valid) return;
    const int wid = 0, lane = threadIdx.x & 31;
    float(*pr)[WROW] = spr[wid];
    float(*qr)[WROW] = sqr[wid];
    float(*stg)[NF][WROW] = sstg[wid];
    float(*bur)[WROW] = sbu[wid];
    const int c0 = sp.x0 + 4 * lane, o0 = WH + 4 * lane;
    const bool edge = lane == 0 || lane == 31;
    const int hc = lane == 0 ? sp.x0 - 4 : sp.x0 + WS, ho = lane == 0 ? WH - 4 : WH + WS;
    const int hp = lane == 0 ? sp.x0 - 8 : sp.x0 + WS, hpo = lane == 0 ? 0 : WH + WS;
    const bool wr = c0 < d.Px, act = c0 < d.Nx;
    for (int k = lane; k < R * WROW; k += 32) (&qr[0][0])[k] = 0.f;
    for (int k = lane; k < 2 * WROW; k += 32) (&bur[0][0])[k] = 0.f;
    const long long so = (long long)sp.s * d.Np;
    const float *A0 = ap0 + so, *AX0 = avx0 + so, *AZ0 = avz0 + so, *PN = pn + so;
    float *A1 = ap1 + so, *AX1 = avx1 + so, *AZ1 = avz1 + so, *GK = accK + so, *GX = accBx + so, *GZ = accBz + so;
    auto axat = [&](const float *a, int c) { return (c >= 0 && c < d.Nx) ? ldg4(a + c) : f4(0.f); };
    const float4 axv = axat(mo.ax, c0), axhv = axat(mo.axh, c0);
    const float4 axp0 = edge ? axat(mo.ax, hp) : f4(0.f), axp1 = edge ? axat(mo.ax, hp + 4) : f4(0.f);
    const float4 axhh = edge ? axat(mo.axh, hc) : f4(0.f);
    const int z0 = sp.z0, zend = min(z0 + tz, d.Nz), f0 = z0 - R;
    auto issue = [&](int g) {
        const int f = f0 + g, r = f - M, j = f - R + 1;
        float *prow = pr[g & (WRP - 1)];
        float(*sg)[WROW] = stg[g & (WNS - 1)];
        cp_row4(prow + o0, PN, d, f, c0);
        cp_row4(sg[0] + o0, A0, d, f, c0);
        cp_row4(sg[1] + o0, mo.K, d, f, c0);
        cp_row4(sg[2] + o0, AZ0, d, r, c0);
        cp_row4(sg[3] + o0, mo.bz, d, r, c0);
        cp_row4(sg[4] + o0, AX0, d, j, c0);
        cp_row4(sg[5] + o0, mo.bx, d, j, c0);
        cp_row4(sg[6] + o0, A0, d, j, c0);
        if (edge) {
            cp_row4(prow + hpo, PN, d, f, hp);
            cp_row4(prow + hpo + 4, PN, d, f, hp + 4);
            cp_row4(sg[0] + hpo, A0, d, f, hp);
            cp_row4(sg[0] + hpo + 4, A0, d, f, hp + 4);
            cp_row4(sg[1] + hpo, mo.K, d, f, hp);
            cp_row4(sg[1] + hpo + 4, mo.K, d, f, hp + 4);
            cp_row4(sg[4] + ho, AX0, d, j, hc);
            cp_row4(sg[5] + ho, mo.bx, d, j, hc);
        }
        cp_commit();
    };
    // qq: K d_p pbar rows f-2M+1 .. f (z-stencil of u_z); bq: bz u_z rows r-2M+1 .. r (z-stencil of
    // pbar); oldest first, shifted every row
    float4 qq[R], bq[R];
#pragma unroll
    for (int k = 0; k < R; ++k) { qq[k] = f4(0.f); bq[k] = f4(0.f); }
#pragma unroll
    for (int g = 0; g < WPD; ++g) issue(g);
    const int fend = zend + R - 1;
#pragma unroll 1
    for (int f = f0; f < fend; ++f) {
        {
            const int g = f - f0, u = f & 1;
            __syncwarp();
            issue(g + WPD);
            cp_wait<WPD>();
            __syncwarp();
            float(*sg)[WROW] = stg[g & (WNS - 1)];
            // q row f = K d_p pbar^{n+1} (own float4; lanes 0/31 also the two halo float4)
            const float azf = (f >= 0 && f < d.Nz) ? __ldg(mo.az + f) : 0.f;
            const float4 qf = (azf * axv) * ld4(sg[1] + o0) * ld4(sg[0] + o0);
#pragma unroll
            for (int q = 0; q < R - 1; ++q) qq[q] = qq[q + 1];
            qq[R - 1] = qf;
            float *qrow = qr[g & (R - 1)];
            st4(qrow + o0, qf);
            if (edge) {
                st4(qrow + hpo, (azf * axp0) * ld4(sg[1] + hpo) * ld4(sg[0] + hpo));
                st4(qrow + hpo + 4, (azf * axp1) * ld4(sg[1] + hpo + 4) * ld4(sg[0] + hpo + 4));
            }
            // u_z at half node r + 1/2, r = f - M
            const int r = f - M;
            float4 gq = f4(0.f), gp = f4(0.f);
#pragma unroll
            for (int k = 1; k <= M; ++k) {   // qq[q] is row f - 2M + 1 + q = r - M + 1 + q
                gq = fma4(st.c[k - 1], qq[M - 1 + k] - qq[M - k], gq);
                gp = fma4(st.c[k - 1], ld4(pr[(g - M + k) & (WRP - 1)] + o0) - ld4(pr[(g - M - k + 1) & (WRP - 1)] + o0), gp);
            }
            const float azh = (r >= 0 && r < d.Nz) ? __ldg(mo.azh + r) : 0.f;
            const float4 uz = mask4((azh * axv) * (ld4(sg[2] + o0) + gq), c0, d.Nx);
#pragma unroll
            for (int q = 0; q < R - 1; ++q) bq[q] = bq[q + 1];
            bq[R - 1] = ld4(sg[3] + o0) * uz;
            if (wr && r >= z0 && r < zend) {
                st4(AZ1 + r * d.Px + c0, uz);
                if (act) red_add4(GZ + r * d.Px + c0, uz * gp);
            }
            // u_x at row j = f - 2M + 1 (own; lanes 0/31 the halo float4 for the divergence)
            const int j = f - R + 1;
            const bool row = j >= z0 && j < zend;
            const float az = (j >= 0 && j < d.Nz) ? __ldg(mo.az + j) : 0.f;
            const int sj = (g - R + 1) & (R - 1), pj = (g - R + 1) & (WRP - 1);
            const float4 ux = mask4((az * axhv) * (ld4(sg[4] + o0) + row_dplus<M>(qr[sj], o0, st)), c0, d.Nx);
            float *brow = bur[u & 1];
            st4(brow + o0, ld4(sg[5] + o0) * ux);
            if (edge) {
                const float4 uh = mask4((az * axhh) * (ld4(sg[4] + ho) + row_dplus<M>(qr[sj], ho, st)), hc, d.Nx);
                st4(brow + ho, hc >= 0 ? ld4(sg[5] + ho) * uh : f4(0.f));
            }
            if (row && wr) {
                st4(AX1 + j * d.Px + c0, ux);
                if (act) red_add4(GX + j * d.Px + c0, ux * row_dplus<M>(pr[pj], o0, st));
            }
            __syncwarp();
            if (row && wr) {
                float4 dv = row_dminus<M>(brow, o0, st);
#pragma unroll
                for (int k = 1; k <= M; ++k)   // bq[q] is row j - M + q
                    dv = fma4(st.c[k - 1], bq[M + k - 1] - bq[M - k], dv);
                const float4 dp = az * axv, a0 = ld4(sg[6] + o0);
                const float4 a1 = mask4(dp * a0 + dv, c0, d.Nx);
                st4(A1 + j * d.Px + c0, a1);
                if (act) red_add4(GK + j * d.Px + c0, ld4(pr[pj] + o0) * (a1 - dp * a0));
            }
        }
    }
    cp_wait<0>();
}

// pbar^{n+1} += R^T r_n at the receivers, and the receiver-cell part of the K-gradient,
// accK += (R^T r_n) p^{n+1} (see k_adj_warp).  One thread per shot and receiver.
__global__ void k_adj_inject_k(float *__restrict__ ap, float *__restrict__ accK, const float *__restrict__ pn1,
                               int ns, int nr, int nt, int n, long long Np, const long long *__restrict__ ridx,
                               const float *__restrict__ rw, const float *__restrict__ res)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns * nr) return;
    const int s = t / nr, r = t - s * nr;
    const float v = res[(long long)t * nt + n];
    const long long so = (long long)s * Np;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const long long o = so + ridx[4 * r + c];
        const float a = rw[4 * r + c] * v;
        atomicAdd(ap + o, a);
        atomicAdd(accK + o, a * pn1[o]);
    }
}

// ------------------------------------------------------------------------ Born (S6)
//
// Background (p, v) and scattered (q, u) fields stepped together, one warp per strip:
//   u^{n+1/2} = d_v (u^{n-1/2} - dt b D+ q^n - dt db D+ p^n)
//   q^{n+1}   = d_p (q^n - dt K D-.u^{n+1/2} - dt dK D-.v^{n+1/2}) + dt dK w_n beta / dx^2
// Rings (with halo) of p and q rows; staged rows (3 stages) of vz, uz, bz, dbz (row f-M) and
// vx, ux, bx, dbx (with halo), K, dK (row j).
template <int M, int MINB>
__global__ void __launch_bounds__(32, MINB) k_born_warp(const float *__restrict__ p0, const float *__restrict__ vx0,
                                                       const float *__restrict__ vz0, const float *__restrict__ q0,
                                                       const float *__restrict__ ux0, const float *__restrict__ uz0,
                                                       float *__restrict__ p1, float *__restrict__ vx1,
                                                       float *__restrict__ vz1, float *__restrict__ q1,
                                                       float *__restrict__ ux1, float *__restrict__ uz1, Model mo,
                                                       Pert pe, Dims d, Stencil st, Source src, int n, int tz,
                                                       int nshots)
{
    constexpr int R = 2 * M, NS = WPD + 1, NF = 10;
    __shared__ __align__(16) float spr[WRP][WROW];
    __shared__ __align__(16) float sqr[WRP][WROW];
    __shared__ __align__(16) float stg[NS][NF][WROW];
    __shared__ __align__(16) float svr[2][WROW];
    __shared__ __align__(16) float sur[2][WROW];
    bool valid;
    const Strip sp = strip_of(d, tz, nshots, valid);
    if (!valid) return;
    const int lane = threadIdx.x & 31;
    const int c0 = sp.x0 + 4 * lane, o0 = WH + 4 * lane;
    const bool edge = lane == 0 || lane == 31;
    const int hc = lane == 0 ? sp.x0 - 4 : sp.x0 + WS, ho = lane == 0 ? WH - 4 : WH + WS;
    const int hp = lane == 0 ? sp.x0 - 8 : sp.x0 + WS, hpo = lane == 0 ? 0 : WH + WS;
    const bool wr = c0 < d.Px, act = c0 < d.Nx;
    const bool hv = edge && hc >= 0 && hc < d.Nx;
    const bool hv0 = edge && hp >= 0 && hp < d.Nx, hv1 = edge && hp + 4 >= 0 && hp + 4 < d.Nx;
    for (int k = lane; k < 2 * WROW; k += 32) { (&svr[0][0])[k] = 0.f; (&sur[0][0])[k] = 0.f; }
    const long long so = (long long)sp.s * d.Np;
    const float *P0 = p0 + so, *VX0 = vx0 + so, *VZ0 = vz0 + so, *Q0 = q0 + so, *UX0 = ux0 + so, *UZ0 = uz0 + so;
    float *P1 = p1 + so, *VX1 = vx1 + so, *VZ1 = vz1 + so, *Q1 = q1 + so, *UX1 = ux1 + so, *UZ1 = uz1 + so;
    const SrcCells sc = src_cells(src, sp.s, d.Px);
    const float wn = __ldg(src.wav + n);
    const float4 axv = act ? ldg4(mo.ax + c0) : f4(0.f), axhv = act ? ldg4(mo.axh + c0) : f4(0.f);
    const float4 axhh = hv ? ldg4(mo.axh + hc) : f4(0.f);
    const int z0 = sp.z0, zend = min(z0 + tz, d.Nz), f0 = z0 - R;
    const bool hsrc = strip_has_src(sc, sp.x0, z0, zend);
    auto issue = [&](int g) {
        const int f = f0 + g, r = f - M, j = f - R + 1;
        const bool vf = f >= 0 && f < d.Nz, vr = r >= 0 && r < d.Nz, vj = j >= 0 && j < d.Nz;
        float *pr = spr[g & (WRP - 1)], *qr = sqr[g & (WRP - 1)];
        float(*sg)[WROW] = stg[g % NS];
        const int of = f * d.Px, orr = r * d.Px, oj = j * d.Px;
        cp16(pr + o0, P0 + of + c0, vf && act);
        cp16(qr + o0, Q0 + of + c0, vf && act);
        cp16(sg[0] + o0, VZ0 + orr + c0, vr && act);
        cp16(sg[1] + o0, UZ0 + orr + c0, vr && act);
        cp16(sg[2] + o0, mo.bz + orr + c0, vr && act);
        cp16(sg[3] + o0, pe.dbz + orr + c0, vr && act);
        cp16(sg[4] + o0, VX0 + oj + c0, vj && act);
        cp16(sg[5] + o0, UX0 + oj + c0, vj && act);
        cp16(sg[6] + o0, mo.bx + oj + c0, vj && act);
        cp16(sg[7] + o0, pe.dbx + oj + c0, vj && act);
        cp16(sg[8] + o0, mo.K + oj + c0, vj && act);
        cp16(sg[9] + o0, pe.dK + oj + c0, vj && act);
        if (edge) {
            cp16(pr + hpo, P0 + of + hp, vf && hv0);
            cp16(pr + hpo + 4, P0 + of + hp + 4, vf && hv1);
            cp16(qr + hpo, Q0 + of + hp, vf && hv0);
            cp16(qr + hpo + 4, Q0 + of + hp + 4, vf && hv1);
            cp16(sg[4] + ho, VX0 + oj + hc, vj && hv);
            cp16(sg[5] + ho, UX0 + oj + hc, vj && hv);
            cp16(sg[6] + ho, mo.bx + oj + hc, vj && hv);
            cp16(sg[7] + ho, pe.dbx + oj + hc, vj && hv);
        }
        cp_commit();
    };
    float4 vq[R], uq[R];   // vz and uz rows r-2M+1 .. r, oldest first
#pragma unroll
    for (int k = 0; k < R; ++k) { vq[k] = f4(0.f); uq[k] = f4(0.f); }
#pragma unroll
    for (int g = 0; g < WPD; ++g) issue(g);
    const int fend = zend + R - 1;
#pragma unroll 1
    for (int f = f0; f < fend; ++f) {
        const int g = f - f0, u = f & 1;
        __syncwarp();
        issue(g + WPD);
        cp_wait<WPD>();
        __syncwarp();
        float(*sg)[WROW] = stg[g % NS];
        const int r = f - M;
        float4 gp = f4(0.f), gq = f4(0.f);
#pragma unroll
        for (int k = 1; k <= M; ++k) {
            const int a = (g - M + k) & (WRP - 1), b = (g - M - k + 1) & (WRP - 1);
            gp = fma4(st.c[k - 1], ld4(spr[a] + o0) - ld4(spr[b] + o0), gp);
            gq = fma4(st.c[k - 1], ld4(sqr[a] + o0) - ld4(sqr[b] + o0), gq);
        }
        const float azh = (r >= 0 && r < d.Nz) ? __ldg(mo.azh + r) : 0.f;
        const float4 fz = azh * axv, bz = ld4(sg[2] + o0);
        const float4 vz = mask4(fz * (ld4(sg[0] + o0) - bz * gp), c0, d.Nx);
        const float4 uz = mask4(fz * (ld4(sg[1] + o0) - bz * gq - ld4(sg[3] + o0) * gp), c0, d.Nx);
        if (wr && r >= z0 && r < zend) {
            st4(VZ1 + r * d.Px + c0, vz);
            st4(UZ1 + r * d.Px + c0, uz);
        }
#pragma unroll
        for (int q = 0; q < R - 1; ++q) { vq[q] = vq[q + 1]; uq[q] = uq[q + 1]; }
        vq[R - 1] = vz;
        uq[R - 1] = uz;
        const int j = f - R + 1;
        const bool row = j >= z0 && j < zend;
        const float az = (j >= 0 && j < d.Nz) ? __ldg(mo.az + j) : 0.f;
        const int sj = (g - R + 1) & (WRP - 1);
        const float *prow = spr[sj], *qrow = sqr[sj];
        const float4 fx = az * axhv, bx = ld4(sg[6] + o0);
        const float4 gpx = row_dplus<M>(prow, o0, st);
        const float4 vx = mask4(fx * (ld4(sg[4] + o0) - bx * gpx), c0, d.Nx);
        const float4 ux = mask4(fx * (ld4(sg[5] + o0) - bx * row_dplus<M>(qrow, o0, st) - ld4(sg[7] + o0) * gpx), c0, d.Nx);
        float *vrow = svr[u], *urow = sur[u];
        st4(vrow + o0, vx);
        st4(urow + o0, ux);
        if (edge) {
            const float4 fh = az * axhh, bh = ld4(sg[6] + ho), gph = row_dplus<M>(prow, ho, st);
            const float4 vh = fh * (ld4(sg[4] + ho) - bh * gph);
            const float4 uh = fh * (ld4(sg[5] + ho) - bh * row_dplus<M>(qrow, ho, st) - ld4(sg[7] + ho) * gph);
            st4(vrow + ho, hv ? mask4(vh, hc, d.Nx) : f4(0.f));
            st4(urow + ho, hv ? mask4(uh, hc, d.Nx) : f4(0.f));
        }
        if (row && wr) {
            st4(VX1 + j * d.Px + c0, vx);
            st4(UX1 + j * d.Px + c0, ux);
        }
        __syncwarp();
        if (row && wr) {
            float4 dv = row_dminus<M>(vrow, o0, st), du = row_dminus<M>(urow, o0, st);
#pragma unroll
            for (int k = 1; k <= M; ++k) {   // vq[q] is vz row j - M + q
                dv = fma4(st.c[k - 1], vq[M + k - 1] - vq[M - k], dv);
                du = fma4(st.c[k - 1], uq[M + k - 1] - uq[M - k], du);
            }
            const float4 K = ld4(sg[8] + o0), dK = ld4(sg[9] + o0), fp = az * axv;
            float4 pn = fp * (ld4(prow + o0) - K * dv);
            float4 qn = fp * (ld4(qrow + o0) - K * du - dK * dv);
            if (hsrc) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (sc.j[k] == j && sc.i[k] >= c0 && sc.i[k] < c0 + 4) {
                        const int c = sc.i[k] - c0;
                        addc(pn, c, comp(K, c) * wn * sc.w[k]);
                        addc(qn, c, comp(dK, c) * wn * sc.w[k]);
                    }
            }
            st4(P1 + j * d.Px + c0, mask4(pn, c0, d.Nx));
            st4(Q1 + j * d.Px + c0, mask4(qn, c0, d.Nx));
        }
    }
    cp_wait<0>();
}

}  // namespace fwi
