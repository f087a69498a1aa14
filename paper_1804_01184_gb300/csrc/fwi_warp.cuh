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
    Strip st;
    st.x0 = (w % nxs) * WS;
    st.z0 = ((w / nxs) % nzs) * tz;
    st.s = w / (nxs * nzs);
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

template <int M, int MINB>
__global__ void __launch_bounds__(64, MINB) k_fwd_warp(const float *__restrict__ p0, const float *__restrict__ vx0,
                                                const float *__restrict__ vz0, float *__restrict__ p1,
                                                float *__restrict__ vx1, float *__restrict__ vz1, Model mo,
                                                Dims d, Stencil st, Source src, int n, int tz, int nshots)
{
    constexpr int R = 2 * M, RP = R + WPD, NS = WPD + 1;
    // per warp: p ring (own + halo columns), staged rows of vz, bz (row f-M) and vx, bx, K (row j)
    __shared__ __align__(16) float sring[2][RP][WROW];
    __shared__ __align__(16) float sstg[2][NS][5][WROW];
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
    const bool wr = c0 < d.Px;
    for (int k = lane; k < 2 * WROW; k += 32) (&vxr[0][0])[k] = 0.f;
    const long long so = (long long)sp.s * d.Np;
    const float *P0 = p0 + so, *VX0 = vx0 + so, *VZ0 = vz0 + so;
    float *P1 = p1 + so, *VX1 = vx1 + so, *VZ1 = vz1 + so;
    const SrcCells sc = src_cells(src, sp.s, d.Px);
    const float wn = __ldg(src.wav + n);
    const float4 axv = c0 < d.Nx ? ldg4(mo.ax + c0) : f4(0.f), axhv = c0 < d.Nx ? ldg4(mo.axh + c0) : f4(0.f);
    const float4 axhh = edge && hc >= 0 && hc < d.Nx ? ldg4(mo.axh + hc) : f4(0.f);
    const int z0 = sp.z0, zend = min(z0 + tz, d.Nz), f0 = z0 - R;
    // stage g: p row f0+g into ring[g % RP]; vz, bz row f0+g-M and vx, bx, K row f0+g-2M+1 into stg[g % NS]
    auto issue = [&](int g) {
        const int f = f0 + g, r = f - M, j = f - R + 1;
        float *pr = ring[g % RP];
        float(*sg)[WROW] = stg[g % NS];
        cp_row4(pr + o0, P0, d, f, c0);
        cp_row4(sg[0] + o0, VZ0, d, r, c0);
        cp_row4(sg[1] + o0, mo.bz, d, r, c0);
        cp_row4(sg[2] + o0, VX0, d, j, c0);
        cp_row4(sg[3] + o0, mo.bx, d, j, c0);
        cp_row4(sg[4] + o0, mo.K, d, j, c0);
        if (edge) {
            cp_row4(pr + hpo, P0, d, f, hp);
            cp_row4(pr + hpo + 4, P0, d, f, hp + 4);
            cp_row4(sg[2] + ho, VX0, d, j, hc);
            cp_row4(sg[3] + ho, mo.bx, d, j, hc);
        }
        cp_commit();
    };
    float4 vq[R];   // vz queue; the p rows of the z-stencil are read from the shared ring
#pragma unroll
    for (int k = 0; k < R; ++k) vq[k] = f4(0.f);
#pragma unroll
    for (int g = 0; g < WPD; ++g) issue(g);
    for (int fb = f0; fb < zend + R - 1; fb += R) {
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int f = fb + u, g = f - f0;
            __syncwarp();                 // every lane is done with the slots issue() refills
            issue(g + WPD);
            cp_wait<WPD>();               // stage g has landed (for this lane)
            __syncwarp();                 // ... and for every lane
            float(*sg)[WROW] = stg[g % NS];
            // vz at half node r + 1/2, r = f - M: p rows r-M+1 .. r+M = stages g-2M+1 .. g
            const int r = f - M;
            float4 gz = f4(0.f);
#pragma unroll
            for (int k = 1; k <= M; ++k)
                gz = fma4(st.c[k - 1], ld4(ring[(g - M + k + 2 * RP) % RP] + o0) -
                                           ld4(ring[(g - M - k + 1 + 2 * RP) % RP] + o0), gz);
            const float azh = (r >= 0 && r < d.Nz) ? __ldg(mo.azh + r) : 0.f;
            const float4 vz = mask4((azh * axv) * (ld4(sg[0] + o0) - ld4(sg[1] + o0) * gz), c0, d.Nx);
            if (wr && r >= z0 && r < zend) st4(VZ1 + r * d.Px + c0, vz);
            vq[u] = vz;
            // v_x at row j = f - 2M + 1 (own float4 and, on lanes 0/31, the halo float4)
            const int j = f - R + 1;
            const bool row = j >= z0 && j < zend;
            const float az = (j >= 0 && j < d.Nz) ? __ldg(mo.az + j) : 0.f;
            const float *prow = ring[(g - R + 1 + RP) % RP];
            const float4 vx = mask4((az * axhv) * (ld4(sg[2] + o0) - ld4(sg[3] + o0) * row_dplus<M>(prow, o0, st)), c0, d.Nx);
            float *vrow = vxr[u & 1];
            st4(vrow + o0, vx);
            if (edge) {
                const float4 vh = mask4((az * axhh) * (ld4(sg[2] + ho) - ld4(sg[3] + ho) * row_dplus<M>(prow, ho, st)), hc, d.Nx);
                st4(vrow + ho, hc >= 0 ? vh : f4(0.f));
            }
            if (row && wr) st4(VX1 + j * d.Px + c0, vx);
            __syncwarp();
            if (row && wr) {
                float4 dv = row_dminus<M>(vrow, o0, st);
#pragma unroll
                for (int k = 1; k <= M; ++k)
                    dv = fma4(st.c[k - 1], vq[(u - M + k + 2 * R) % R] - vq[(u + 1 - k - M + 2 * R) % R], dv);
                const float4 Kv = ld4(sg[4] + o0);
                float4 pn = (az * axv) * (ld4(prow + o0) - Kv * dv);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (sc.j[k] == j && sc.i[k] >= c0 && sc.i[k] < c0 + 4)
                        addc(pn, sc.i[k] - c0, comp(Kv, sc.i[k] - c0) * wn * sc.w[k]);
                st4(P1 + j * d.Px + c0, mask4(pn, c0, d.Nx));
            }
        }
    }
    cp_wait<0>();
}

}  // namespace fwi
