// fwi_warp.cuh -- warp-strip streaming time-step kernels (sm_103a).
//
// Every warp owns a strip of WS = 120 columns of one shot (lanes 0..29, a float4 each) and
// tz rows, and marches down it alone: no block barriers, one __syncwarp pair per row.
//   - Lanes 30 and 31 carry the strip's x-halo in the same instruction stream: lane 30 the
//     float4 left of the strip (x0-4) and lane 31 the one right of it (x0+120), each with one
//     more pressure float4 (x0-8, x0+124).  They compute the v_x halo values the divergence of
//     the strip's edge columns needs, so no lane ever runs a divergent halo branch.
//   - z-neighbours: shared rings of p-like rows (2M + the prefetch depth) and a register queue
//     of v_z rows.
//   - x-neighbours: a shared row (columns x0-8 .. x0+127) per field.
//   - Global rows arrive by 16-byte cp.async (zero-filled outside the grid) FWD_WPD, ADJ_WPD
//     or BORN_WPD rows ahead.
//   - Element-wise updates and z-stencils use packed FP32x2 arithmetic.
// Every value outside the computational grid is zero: the model and sponge arrays are zero in
// the padding columns, so every update there is exactly zero; every own lane whose float4
// starts below the row pitch writes it, so written rows are fully defined.
#pragma once
#include "fwi_stream.cuh"

namespace fwi {

constexpr int WS = 120;    // columns owned by a warp
constexpr int WH = 8;      // shared offset of column x0
constexpr int WROW = 136;  // shared row: columns x0-8 .. x0+127
// rows each family prefetches ahead (measured on GB300: deeper staging costs shared memory,
// hence resident warps; these depths balance the two)
constexpr int FWD_WPD = 3;
constexpr int ADJ_WPD = 3;
constexpr int BORN_WPD = 2;
constexpr int FWD_WPB = 2; // warps per block of the forward kernels

// Slot of row g + c in a ring of N rows, for the row g the loop is at (|c| < N); the ring
// position of g advances by one per row, so no division is needed.
template <int N>
struct RingPos {
    int b = 0;   // g mod N
    __device__ __forceinline__ int operator()(int c) const
    {
        int s = b + c;
        if (c < 0) s += s < 0 ? N : 0;
        if (c > 0) s -= s >= N ? N : 0;
        return s;
    }
    __device__ __forceinline__ void next() { b = b + 1 == N ? 0 : b + 1; }
};

// The streaming kernels keep their per-warp staging in dynamic shared memory (deep stagings
// exceed the 48 KB static limit); fwd_smem<M>(), adj_smem<M>() and born_smem<M>() give the bytes
// per block.

struct Strip {
    int x0, z0, s;      // strip origin and shot
};

// Warps a launch over `nshots` shots of grid d needs.
__host__ __device__ __forceinline__ int strip_warps(const Dims &d, int tz, int nshots)
{
    return ((d.Nx + WS - 1) / WS) * ((d.Nz + tz - 1) / tz) * nshots;
}

// warp w of a launch -> strip; the shot varies fastest so that warps running together stream
// the same model rows (shared by every shot of the launch) and find them in L1/L2
__device__ __forceinline__ Strip strip_at(int w, const Dims &d, int tz, int nshots, bool &valid)
{
    const int nxs = (d.Nx + WS - 1) / WS;
    valid = w < strip_warps(d, tz, nshots);
    Strip st;
    st.s = w % nshots;
    st.x0 = ((w / nshots) % nxs) * WS;
    st.z0 = (w / (nshots * nxs)) * tz;
    return st;
}

__device__ __forceinline__ Strip strip_of(const Dims &d, int tz, int nshots, int wpb, bool &valid)
{
    return strip_at(blockIdx.x * wpb + (threadIdx.x >> 5), d, tz, nshots, valid);
}

// Batched launches carry their job table as a kernel parameter (__grid_constant__, at most
// 32 KB): warp (or thread) w belongs to job j with wstart[j] <= w < wstart[j+1].
constexpr int BATCH_CAP = 96;

template <typename A>
struct BatchTable {
    int njobs;
    int wstart[BATCH_CAP + 1];
    A jobs[BATCH_CAP];
};

__device__ __forceinline__ int job_of(int w, const int *wstart, int njobs, int &local)
{
    int lo = 0, hi = njobs;          // invariant: wstart[lo] <= w < wstart[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (wstart[mid] <= w) lo = mid; else hi = mid;
    }
    local = w - wstart[lo];
    return lo;
}

// Role of a lane: its main float4 (own column, or the halo float4 for lanes 30/31) and, on the
// halo lanes, one extra pressure float4.
struct LaneMap {
    int mc, mo;         // main column and its shared offset
    int ec, eo;         // extra column / offset (halo lanes)
    bool own;           // lanes 0..29
    bool in, ein;       // main / extra float4 inside the grid
    bool wr;            // own and below the row pitch: writes global rows
};

__device__ __forceinline__ LaneMap lane_map(int lane, int x0, const Dims &d)
{
    LaneMap m;
    m.own = lane < 30;
    m.mc = m.own ? x0 + 4 * lane : (lane == 30 ? x0 - 4 : x0 + WS);
    m.ec = lane == 30 ? x0 - 8 : x0 + WS + 4;
    m.mo = m.mc - x0 + WH;
    m.eo = m.ec - x0 + WH;
    m.in = m.mc >= 0 && m.mc < d.Nx;
    m.ein = !m.own && m.ec >= 0 && m.ec < d.Nx;
    m.wr = m.own && m.mc < d.Px;
    return m;
}

// 16-byte asynchronous copy of base[off .. off+3] into shared dst, zero-filled when !valid; an
// invalid copy reads nothing and is given the (valid) base address, never base + off
__device__ __forceinline__ void cp16(void *dst, const float *base, int off, bool valid)
{
    const float *src = base + (valid ? off : 0);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
// 4-byte asynchronous copy of base[off] (zero when !valid), as cp16
__device__ __forceinline__ void cp4(void *dst, const float *base, int off, bool valid)
{
    const float *src = base + (valid ? off : 0);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// fire-and-forget vector add into global memory (resolved in L2; one warp owns each address
// within a launch, so the order of additions is fixed)
__device__ __forceinline__ void red_add4(float *dst, float4 v)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// Does the strip hold any source cell of its shot? (uniform per warp)
__device__ __forceinline__ bool strip_has_src(const SrcCells &sc, int x0, int z0, int zend)
{
    bool h = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) h |= sc.i[k] >= x0 && sc.i[k] < x0 + WS && sc.j[k] >= z0 && sc.j[k] < zend;
    return h;
}

__device__ __forceinline__ float4 ldg_if(const float *p, bool v) { return v ? ldg4(p) : f4(0.f); }

// Trace sampling of the PREVIOUS step carried by a single-job launch: the launch reads that
// step's field (p^n, or the scattered q^n) only as its input, so extra warps appended to the
// grid can sample it while the strips compute the next step; one launch fewer per step.
// trace[s][r][n - 1] = sum_c beta_rc field[cell_rc], in the same corner order as k_sample.
struct Tail {
    const float *field;           // [shots][Np] the launch's input field
    float *traces;                // [shots][nr][nt]
    const long long *ridx;
    const float *rw;
    long long Np;
    int nr, nt, col;              // col: trace sample written (n - 1)
    int count;                    // shots x nr (0: no sampling)
};

__device__ __forceinline__ void sample_tail(const Tail &tl, int t)
{
    if (t >= tl.count) return;
    const int s = t / tl.nr, r = t - s * tl.nr;
    const float *ps = tl.field + (long long)s * tl.Np;
    float v = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (FWI_IN(true, tl.ridx[4 * r + c], 1, tl.Np, nullptr)) v += tl.rw[4 * r + c] * ps[tl.ridx[4 * r + c]];
    tl.traces[(long long)t * tl.nt + tl.col] = v;
}

__host__ __device__ __forceinline__ int tail_warps(const Tail &tl) { return (tl.count + 31) / 32; }

// ------------------------------------------------------------------ forward step (S3)
//
//   v^{n+1/2} = d_v (v^{n-1/2} - dt b D+ p^n);  p^{n+1} = d_p (p^n - dt K D-.v^{n+1/2}) + dt K w_n beta/dx^2
struct FwdArgs {
    const float *p0, *vx0, *vz0;    // p^n, v^{n-1/2} of the launch's shots
    float *p1, *vx1, *vz1;          // p^{n+1}, v^{n+1/2}
    Model mo;
    Dims d;
    Stencil st;
    Source src;                     // sources of the launch's shots
    int n, tz, nshots;
};

// Shared memory of one warp of a forward launch (2M + FWD_WPD pressure rows: the 2M the stencils
// read and the FWD_WPD in flight; FWD_WPD + 1 stages).
template <int M>
struct FwdSmem {
    float ring[2 * M + FWD_WPD][WROW];  // p^n rows
    float stg[FWD_WPD + 1][5][WROW];    // vz, bz (row f-M); vx, bx, K (row j)
    float vxr[2][WROW];             // v_x^{n+1/2} rows
    float scl[FWD_WPD + 1][4];          // az(j), azh(r) of each stage
};

template <int M>
__device__ __forceinline__ void fwd_body(const FwdArgs &a, const Strip &sp, FwdSmem<M> &sh)
{
    constexpr int R = 2 * M, NP = 2 * M + FWD_WPD, NS = FWD_WPD + 1;
    const Dims &d = a.d;
    const Model &mo = a.mo;
    const Stencil &st = a.st;
    const int n = a.n, tz = a.tz;
    const int lane = threadIdx.x & 31;
    float(*ring)[WROW] = sh.ring;
    float(*stg)[5][WROW] = sh.stg;
    float(*vxr)[WROW] = sh.vxr;
    const LaneMap L = lane_map(lane, sp.x0, d);
    for (int k = lane; k < 2 * WROW; k += 32) (&vxr[0][0])[k] = 0.f;
    const long long so = (long long)sp.s * d.Np;
    const float *P0 = a.p0 + so, *VX0 = a.vx0 + so, *VZ0 = a.vz0 + so;
    float *P1 = a.p1 + so, *VX1 = a.vx1 + so, *VZ1 = a.vz1 + so;
    const SrcCells sc = src_cells(a.src, sp.s, d.Px);
    const float wn = __ldg(a.src.wav + n);
    const float4 axv = ldg_if(mo.ax + L.mc, L.in), axhv = ldg_if(mo.axh + L.mc, L.in);
    const int z0 = sp.z0, zend = min(z0 + tz, d.Nz), f0 = z0 - R;
    const bool hsrc = strip_has_src(sc, sp.x0, z0, zend);
    // stage row g (rows f = f0 + g; r = f - M; j = f - 2M + 1) into ring slot ps, stage ss
    // rows the strip's outputs depend on (the others stream in as zeros, reading nothing):
    // p rows f >= z0 - 2M + 1, v_z rows r >= z0 - M, v_x / model rows j >= z0
    auto issue = [&](int g, int ps, int ss) {
        const int f = f0 + g, r = f - M, j = f - R + 1;
        const bool vf = f >= max(0, z0 - R + 1) && f < d.Nz, vr = r >= max(0, z0 - M) && r < d.Nz,
                   vj = j >= z0 && j < d.Nz;
        float *pr = ring[ps];
        float(*sg)[WROW] = stg[ss];
        const int of = f * d.Px, orr = r * d.Px, oj = j * d.Px;
        const long long np = d.Np;
        int *stt = mo.status;
        cp16(pr + L.mo, P0, of + L.mc, FWI_IN(vf && L.in, of + L.mc, 4, np, stt));
        if (!L.own) cp16(pr + L.eo, P0, of + L.ec, FWI_IN(vf && L.ein, of + L.ec, 4, np, stt));
        const bool zo = FWI_IN(vr && L.in && L.own, orr + L.mc, 4, np, stt);
        cp16(sg[0] + L.mo, VZ0, orr + L.mc, zo);
        cp16(sg[1] + L.mo, mo.bz, orr + L.mc, zo);
        const bool xo = FWI_IN(vj && L.in, oj + L.mc, 4, np, stt);
        cp16(sg[2] + L.mo, VX0, oj + L.mc, xo);
        cp16(sg[3] + L.mo, mo.bx, oj + L.mc, xo);
        cp16(sg[4] + L.mo, mo.K, oj + L.mc, xo && L.own);
        if (lane == 0) {
            cp4(&sh.scl[ss][0], mo.az, j, FWI_IN(vj, j, 1, d.Nz, stt));
            cp4(&sh.scl[ss][1], mo.azh, r, FWI_IN(vr, r, 1, d.Nz, stt));
        }
        cp_commit();
    };
    float4 vq[R];   // vz rows r-2M+1 .. r (oldest first), shifted every row
    float4 pq[R];   // this lane's own p float4 of rows g-2M+1 .. g (oldest first): the z-stencil
                    // reads registers instead of 2M shared rows
#pragma unroll
    for (int k = 0; k < R; ++k) vq[k] = pq[k] = f4(0.f);
#pragma unroll
    for (int g = 0; g < FWD_WPD; ++g) issue(g, g, g);
    RingPos<NP> P;      // ring position of row g
    RingPos<NS> S;      // stage of row g
    const int fend = zend + R - 1;
#pragma unroll 2   // two rows per trip: half the register-queue shifts (measured: 1 < 2 > 4)
    for (int f = f0; f < fend; ++f) {
        const int g = f - f0;
        __syncwarp();                 // every lane is done with the slots issue() refills
        issue(g + FWD_WPD, P(FWD_WPD), S(FWD_WPD));
        cp_wait<FWD_WPD>();               // stage g has landed (for this lane) ...
        __syncwarp();                 // ... and for every lane
        float(*sg)[WROW] = stg[S(0)];
        const float az = sh.scl[S(0)][0], azh = sh.scl[S(0)][1];
        // vz at half node r + 1/2, r = f - M: p rows r-M+1 .. r+M = rows g-2M+1 .. g
        const int r = f - M;
#pragma unroll
        for (int q = 0; q < R - 1; ++q) pq[q] = pq[q + 1];
        pq[R - 1] = ld4(ring[P(0)] + L.mo);
        float4 gz = f4(0.f);          // -dt D+z p (pq[q] is row g - 2M + 1 + q)
#pragma unroll
        for (int k = 1; k <= M; ++k)
            gz = ptap(st.nc[k - 1], pq[M - 1 + k], pq[M - k], gz);
        const float4 vz = pmul(pmul(azh, axv), pfma(ld4(sg[1] + L.mo), gz, ld4(sg[0] + L.mo)));
        if (FWI_IN(L.wr && r >= z0 && r < zend, (long long)r * d.Px + L.mc, 4, d.Np, mo.status))
            st4(VZ1 + r * d.Px + L.mc, vz);
#pragma unroll
        for (int q = 0; q < R - 1; ++q) vq[q] = vq[q + 1];
        vq[R - 1] = vz;
        // v_x at row j = f - 2M + 1 (every lane: own columns and the two halo float4)
        const int j = f - R + 1;
        const bool row = j >= z0 && j < zend;
        const float *prow = ring[P(1 - R)];
        const float4 gx = row_dplus<M>(prow, L.mo, pq[0], st.nc);        // -dt D+x p
        const float4 vx = pmul(pmul(az, axhv), pfma(ld4(sg[3] + L.mo), gx, ld4(sg[2] + L.mo)));
        float *vrow = vxr[f & 1];
        st4(vrow + L.mo, vx);
        const bool jw = FWI_IN(row && L.wr, (long long)j * d.Px + L.mc, 4, d.Np, mo.status);
        if (jw) st4(VX1 + j * d.Px + L.mc, vx);
        __syncwarp();
        if (jw) {
            float4 dv = row_dminus<M>(vrow, L.mo, vx, st.nc);          // -dt D-x vx
#pragma unroll
            for (int k = 1; k <= M; ++k)   // vq[q] is vz row j - M + q
                dv = ptap(st.nc[k - 1], vq[M + k - 1], vq[M - k], dv);
            const float4 Kv = ld4(sg[4] + L.mo);
            float4 pn = pmul(pmul(az, axv), pfma(Kv, dv, pq[0]));
            if (hsrc) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (sc.j[k] == j && sc.i[k] >= L.mc && sc.i[k] < L.mc + 4)
                        addc(pn, sc.i[k] - L.mc, comp(Kv, sc.i[k] - L.mc) * wn * sc.w[k]);
            }
            st4(P1 + j * d.Px + L.mc, pn);
        }
        P.next();
        S.next();
    }
    cp_wait<0>();
}

// MINB: blocks per SM the register budget is sized for (1: unbounded); minb() gives the
// MINB that caps a block of `threads` threads at `regs` registers a thread
constexpr int minb(int regs, int threads) { return 65536 / (regs * threads); }

template <int M, int MINB>
__global__ void __launch_bounds__(32 * FWD_WPB, MINB) k_fwd_warp(FwdArgs a, Tail tl)
{
    extern __shared__ __align__(16) unsigned char fwi_smem[];
    const int w = blockIdx.x * FWD_WPB + (threadIdx.x >> 5), nw = strip_warps(a.d, a.tz, a.nshots);
    if (w >= nw) {   // a sampling warp
        sample_tail(tl, (w - nw) * 32 + (threadIdx.x & 31));
        return;
    }
    bool valid;
    const Strip sp = strip_at(w, a.d, a.tz, a.nshots, valid);
    fwd_body<M>(a, sp, reinterpret_cast<FwdSmem<M> *>(fwi_smem)[threadIdx.x >> 5]);
}

// Per-receiver work of the batching engine that rides on a batched forward launch after its
// strips: trace samples of the previous engine iteration's steps (their fields are final and
// only read in this launch) and this iteration's adjoint injections (their fields are read
// by a later launch).  Thread u of the tail takes sample unit u, then injection units.
struct SampleItem {
    const float *p;            // p^{n+1} (or q^{n+1}) of the job's group
    float *traces;             // [bg][nr][nt] of the group
    const long long *ridx;
    const float *rw;
    long long Np;
    int bg, nr, nt, n;
};

struct InjectItem {
    float *ap, *accK;
    const float *pn1, *res;
    const long long *ridx;
    const float *rw;
    const int *rl;
    long long Np;
    int bg, nr, nt, n;
};

constexpr int SMALL_CAP = 40;

struct SmallTable {
    int nsmp, ninj;
    int smp_start[SMALL_CAP + 1];     // prefix counts of units (threads)
    int inj_start[SMALL_CAP + 1];
    SampleItem smp[SMALL_CAP];
    InjectItem inj[SMALL_CAP];
};

// defined with the adjoint kernels below
__device__ __forceinline__ void inject_entry(float *__restrict__ ap, float *__restrict__ accK,
                                             const float *__restrict__ pn1, int s, int k, int nr, int nt, int n,
                                             long long Np, const long long *__restrict__ ridx,
                                             const float *__restrict__ rw, const int *__restrict__ rl,
                                             const float *__restrict__ res);

__device__ __forceinline__ int small_units(const SmallTable &s) { return s.smp_start[s.nsmp] + s.inj_start[s.ninj]; }

__device__ __forceinline__ void small_work(const SmallTable &s, int u)
{
    const int ns = s.smp_start[s.nsmp];
    int l;
    if (u < ns) {
        const SampleItem &d = s.smp[job_of(u, s.smp_start, s.nsmp, l)];
        const int sh = l / d.nr, r = l - sh * d.nr;
        const float *ps = d.p + (long long)sh * d.Np;
        float v = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (FWI_IN(true, d.ridx[4 * r + c], 1, d.Np, nullptr)) v += d.rw[4 * r + c] * ps[d.ridx[4 * r + c]];
        d.traces[(long long)l * d.nt + d.n] = v;
        return;
    }
    u -= ns;
    if (u >= s.inj_start[s.ninj]) return;
    const InjectItem &d = s.inj[job_of(u, s.inj_start, s.ninj, l)];
    const int sh = l / (4 * d.nr);
    inject_entry(d.ap, d.accK, d.pn1, sh, l - sh * 4 * d.nr, d.nr, d.nt, d.n, d.Np, d.ridx, d.rw, d.rl, d.res);
}

// A launch of per-receiver work alone (when no forward launch can carry it).
__global__ void k_small_batch(const __grid_constant__ SmallTable s)
{
    small_work(s, blockIdx.x * blockDim.x + threadIdx.x);
}

// One time step of several independent jobs: warp w runs strip (w - wstart[j]) of job j;
// the warps after the strips do the per-receiver work of table s.
template <int M>
__global__ void __launch_bounds__(32 * FWD_WPB) k_fwd_batch(const __grid_constant__ BatchTable<FwdArgs> t,
                                                          const __grid_constant__ SmallTable s)
{
    extern __shared__ __align__(16) unsigned char fwi_smem[];
    const int w = blockIdx.x * FWD_WPB + (threadIdx.x >> 5);
    if (w >= t.wstart[t.njobs]) {
        small_work(s, (w - t.wstart[t.njobs]) * 32 + (threadIdx.x & 31));
        return;
    }
    int local;
    const FwdArgs &a = t.jobs[job_of(w, t.wstart, t.njobs, local)];
    bool valid;
    const Strip sp = strip_at(local, a.d, a.tz, a.nshots, valid);
    if (!valid) return;
    fwd_body<M>(a, sp, reinterpret_cast<FwdSmem<M> *>(fwi_smem)[threadIdx.x >> 5]);
}

// ------------------------------------------------------------- adjoint step (S7)
//
// Reverse step n, the transpose of k_fwd_warp's step, with the cross-correlation fused in:
//   q = K d_p pbar^{n+1};  u = d_v (vbar + dt D+ q) -> new vbar;  pbar^n = d_p pbar^{n+1} + dt D- (b u)
//   accBz/accBx += u dt D+ p^n    (g_b = -accB)
//   accK += p^n (pbar^n - d_p pbar^{n+1}) = p^n dt D- (b u)      (g_K = accK / K)
// The last line pairs each pressure adjoint with its own snapshot one launch earlier than the
// textbook form sum pbar^{n+1} (p^{n+1} - d_p p^n); the receiver-cell remainder
// (R^T r_n) p^{n+1} is added by k_adj_inject_k.
struct AdjArgs {
    const float *ap0, *avx0, *avz0;   // pbar^{n+1} (after injection), vbar^{n+1/2}
    float *ap1, *avx1, *avz1;         // pbar^n, new vbar
    Model mo;
    const float *pn;                  // p^n snapshots of the launch's shots
    float *accK, *accBx, *accBz;      // FP32 gradient accumulators of the launch's shots
    Dims d;
    Stencil st;
    int tz, nshots;
};

// Shared memory of one adjoint warp.
template <int M>
struct AdjSmem {
    float pr[2 * M + ADJ_WPD][WROW];      // p^n rows
    float qr[2 * M][WROW];            // K d_p pbar^{n+1} rows
    float stg[ADJ_WPD + 1][7][WROW];      // pbar, K (row f); vbar_z, bz (row r); vbar_x, bx, pbar (row j)
    float bur[2][WROW];               // bx u_x rows
    float scl[ADJ_WPD + 1][4];            // az(f), azh(r), az(j) of each stage
};

template <int M>
__device__ __forceinline__ void adj_body(const AdjArgs &a, const Strip &sp, AdjSmem<M> &sh)
{
    constexpr int R = 2 * M, NF = 7, NP = 2 * M + ADJ_WPD, NS = ADJ_WPD + 1;
    const Dims &d = a.d;
    const Model &mo = a.mo;
    const Stencil &st = a.st;
    const int tz = a.tz;
    float(*pr)[WROW] = sh.pr;
    float(*qr)[WROW] = sh.qr;
    float(*stg)[NF][WROW] = sh.stg;
    float(*bur)[WROW] = sh.bur;
    const int lane = threadIdx.x & 31;
    const LaneMap L = lane_map(lane, sp.x0, d);
    for (int k = lane; k < R * WROW; k += 32) (&qr[0][0])[k] = 0.f;
    for (int k = lane; k < 2 * WROW; k += 32) (&bur[0][0])[k] = 0.f;
    const long long so = (long long)sp.s * d.Np;
    const float *A0 = a.ap0 + so, *AX0 = a.avx0 + so, *AZ0 = a.avz0 + so, *PN = a.pn + so;
    float *A1 = a.ap1 + so, *AX1 = a.avx1 + so, *AZ1 = a.avz1 + so;
    float *GK = a.accK + so, *GX = a.accBx + so, *GZ = a.accBz + so;
    const float4 axv = ldg_if(mo.ax + L.mc, L.in), axhv = ldg_if(mo.axh + L.mc, L.in);
    const float4 axe = ldg_if(mo.ax + L.ec, L.ein);
    const int z0 = sp.z0, zend = min(z0 + tz, d.Nz), f0 = z0 - R;
    // rows the strip's outputs depend on (the others stream in as zeros, reading nothing):
    // pbar / K rows f >= z0 - 2M + 1, forward p rows f >= z0 - M + 1, u_z rows r >= z0 - M,
    // u_x rows j >= z0
    auto issue = [&](int g, int ps, int ss) {
        const int f = f0 + g, r = f - M, j = f - R + 1;
        const bool vf = f >= max(0, z0 - R + 1) && f < d.Nz, vr = r >= max(0, z0 - M) && r < d.Nz,
                   vj = j >= z0 && j < d.Nz, vp = vf && f >= z0 - M + 1;
        float *prow = pr[ps];
        float(*sg)[WROW] = stg[ss];
        const int of = f * d.Px, orr = r * d.Px, oj = j * d.Px;
        const long long np = d.Np;
        int *stt = mo.status;
        if (lane == 0) {
            cp4(&sh.scl[ss][0], mo.az, f, FWI_IN(vf, f, 1, d.Nz, stt));
            cp4(&sh.scl[ss][1], mo.azh, r, FWI_IN(vr, r, 1, d.Nz, stt));
            cp4(&sh.scl[ss][2], mo.az, j, FWI_IN(vj, j, 1, d.Nz, stt));
        }
        const bool fm = FWI_IN(vf && L.in, of + L.mc, 4, np, stt);
        cp16(prow + L.mo, PN, of + L.mc, vp && fm);
        cp16(sg[0] + L.mo, A0, of + L.mc, fm);
        cp16(sg[1] + L.mo, mo.K, of + L.mc, fm);
        if (!L.own) {
            const bool fe = FWI_IN(vf && L.ein, of + L.ec, 4, np, stt);
            cp16(prow + L.eo, PN, of + L.ec, vp && fe);
            cp16(sg[0] + L.eo, A0, of + L.ec, fe);
            cp16(sg[1] + L.eo, mo.K, of + L.ec, fe);
        }
        const bool zo = FWI_IN(vr && L.in && L.own, orr + L.mc, 4, np, stt);
        cp16(sg[2] + L.mo, AZ0, orr + L.mc, zo);
        cp16(sg[3] + L.mo, mo.bz, orr + L.mc, zo);
        const bool xo = FWI_IN(vj && L.in, oj + L.mc, 4, np, stt);
        cp16(sg[4] + L.mo, AX0, oj + L.mc, xo);
        cp16(sg[5] + L.mo, mo.bx, oj + L.mc, xo);
        cp16(sg[6] + L.mo, A0, oj + L.mc, xo && L.own);
        cp_commit();
    };
    // qq: K d_p pbar rows f-2M+1 .. f (z-stencil of u_z); bq: bz u_z rows r-2M+1 .. r (z-stencil of
    // pbar); oldest first, shifted every row
    float4 qq[R], bq[R];
    float4 pq[R];   // this lane's own p^n float4 of rows g-2M+1 .. g (z-stencil from registers)
#pragma unroll
    for (int k = 0; k < R; ++k) { qq[k] = f4(0.f); bq[k] = f4(0.f); pq[k] = f4(0.f); }
#pragma unroll
    for (int g = 0; g < ADJ_WPD; ++g) issue(g, g, g);
    RingPos<NP> P;      // ring position of row g in pr
    RingPos<NS> S;      // stage of row g
    RingPos<R> Q;       // ring position of row g in qr
    const int fend = zend + R - 1;
#pragma unroll 2   // two rows per trip: half the register-queue shifts (measured: 1 < 2 > 4)
    for (int f = f0; f < fend; ++f) {
        const int g = f - f0;
        __syncwarp();
        issue(g + ADJ_WPD, P(ADJ_WPD), S(ADJ_WPD));
        cp_wait<ADJ_WPD>();
        __syncwarp();
        float(*sg)[WROW] = stg[S(0)];
        const float azf = sh.scl[S(0)][0], azh = sh.scl[S(0)][1], az = sh.scl[S(0)][2];
        // q row f = K d_p pbar^{n+1} (main float4; halo lanes also the extra float4)
        const float4 qf = pmul(pmul(azf, axv), pmul(ld4(sg[1] + L.mo), ld4(sg[0] + L.mo)));
#pragma unroll
        for (int q = 0; q < R - 1; ++q) qq[q] = qq[q + 1];
        qq[R - 1] = qf;
        float *qrow = qr[Q(0)];
        st4(qrow + L.mo, qf);
        if (!L.own) st4(qrow + L.eo, pmul(pmul(azf, axe), pmul(ld4(sg[1] + L.eo), ld4(sg[0] + L.eo))));
        // u_z at half node r + 1/2, r = f - M
        const int r = f - M;
#pragma unroll
        for (int q = 0; q < R - 1; ++q) pq[q] = pq[q + 1];
        pq[R - 1] = ld4(pr[P(0)] + L.mo);
        float4 gq = f4(0.f), gp = f4(0.f);
#pragma unroll
        for (int k = 1; k <= M; ++k) {   // qq[q], pq[q] are row f - 2M + 1 + q = r - M + 1 + q
            gq = ptap(st.c[k - 1], qq[M - 1 + k], qq[M - k], gq);
            gp = ptap(st.c[k - 1], pq[M - 1 + k], pq[M - k], gp);
        }
        const float4 uz = pmul(pmul(azh, axv), padd(ld4(sg[2] + L.mo), gq));
#pragma unroll
        for (int q = 0; q < R - 1; ++q) bq[q] = bq[q + 1];
        bq[R - 1] = pmul(ld4(sg[3] + L.mo), uz);
        if (FWI_IN(L.wr && r >= z0 && r < zend, (long long)r * d.Px + L.mc, 4, d.Np, mo.status)) {
            st4(AZ1 + r * d.Px + L.mc, uz);
            red_add4(GZ + r * d.Px + L.mc, pmul(uz, gp));
        }
        // u_x at row j = f - 2M + 1 (every lane: own columns and the two halo float4)
        const int j = f - R + 1;
        const bool row = j >= z0 && j < zend;
        const float *pj = pr[P(1 - R)];
        const float4 ux = pmul(pmul(az, axhv), padd(ld4(sg[4] + L.mo), row_dplus<M>(qr[Q(1 - R)], L.mo, qq[0], st.c)));
        float *brow = bur[f & 1];
        const float4 bux = pmul(ld4(sg[5] + L.mo), ux);
        st4(brow + L.mo, bux);
        const bool jw = FWI_IN(row && L.wr, (long long)j * d.Px + L.mc, 4, d.Np, mo.status);
        if (jw) {
            st4(AX1 + j * d.Px + L.mc, ux);
            red_add4(GX + j * d.Px + L.mc, pmul(ux, row_dplus<M>(pj, L.mo, pq[0], st.c)));
        }
        __syncwarp();
        if (jw) {
            float4 dv = row_dminus<M>(brow, L.mo, bux, st.c);
#pragma unroll
            for (int k = 1; k <= M; ++k)   // bq[q] is row j - M + q
                dv = ptap(st.c[k - 1], bq[M + k - 1], bq[M - k], dv);
            const float4 dp = pmul(az, axv);
            st4(A1 + j * d.Px + L.mc, pfma(dp, ld4(sg[6] + L.mo), dv));
            // pbar^n - d_p pbar^{n+1} is exactly the divergence term dv
            red_add4(GK + j * d.Px + L.mc, pmul(pq[0], dv));
        }
        P.next();
        S.next();
        Q.next();
    }
    cp_wait<0>();
}

template <int M, int MINB>
__global__ void __launch_bounds__(32, MINB) k_adj_warp(AdjArgs a)
{
    extern __shared__ __align__(16) unsigned char fwi_smem[];   // one warp per block
    bool valid;
    const Strip sp = strip_of(a.d, a.tz, a.nshots, 1, valid);
    if (!valid) return;
    adj_body<M>(a, sp, *reinterpret_cast<AdjSmem<M> *>(fwi_smem));
}

template <int M>
__global__ void __launch_bounds__(32) k_adj_batch(const __grid_constant__ BatchTable<AdjArgs> t)
{
    extern __shared__ __align__(16) unsigned char fwi_smem[];
    AdjSmem<M> &sh = *reinterpret_cast<AdjSmem<M> *>(fwi_smem);
    const int w = blockIdx.x;
    if (w >= t.wstart[t.njobs]) return;
    int local;
    const AdjArgs &a = t.jobs[job_of(w, t.wstart, t.njobs, local)];
    bool valid;
    const Strip sp = strip_at(local, a.d, a.tz, a.nshots, valid);
    if (!valid) return;
    adj_body<M>(a, sp, sh);
}

// pbar^{n+1} += R^T r_n at the receivers, and the receiver-cell part of the K-gradient,
// accK += (R^T r_n) p^{n+1} (see k_adj_warp).  One thread per shot and receiver.
// Injection of receiver footprint k of shot-slot s at step n: the first entry of every cell
// sums the chain of footprints on that cell in receiver order and adds once, so the result
// does not depend on thread order even when receivers share cells.
__device__ __forceinline__ void inject_entry(float *__restrict__ ap, float *__restrict__ accK,
                                             const float *__restrict__ pn1, int s, int k, int nr, int nt, int n,
                                             long long Np, const long long *__restrict__ ridx,
                                             const float *__restrict__ rw, const int *__restrict__ rl,
                                             const float *__restrict__ res)
{
    const int n4 = 4 * nr;
    int m = rl[k];
    if (!(m & CHAIN_FIRST)) return;
    const float *rs = res + (long long)s * nr * nt + n;
    float a = rw[k] * rs[(long long)(k >> 2) * nt];
    for (m &= CHAIN_FIRST - 1; m < n4; m = rl[m] & (CHAIN_FIRST - 1)) a += rw[m] * rs[(long long)(m >> 2) * nt];
    if (!FWI_IN(true, ridx[k], 1, Np, nullptr)) return;
    const long long o = (long long)s * Np + ridx[k];
    ap[o] += a;
    accK[o] += a * pn1[o];
}

// Adds the residual R^T r_n into pbar^{n+1} and the receiver-cell term (R^T r_n) p^{n+1}
// into the K accumulator; one thread per (shot, receiver footprint entry).
__global__ void k_adj_inject_k(float *__restrict__ ap, float *__restrict__ accK, const float *__restrict__ pn1,
                               int ns, int nr, int nt, int n, long long Np, const long long *__restrict__ ridx,
                               const float *__restrict__ rw, const int *__restrict__ rl, const float *__restrict__ res)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns * 4 * nr) return;
    const int s = t / (4 * nr);
    inject_entry(ap, accK, pn1, s, t - s * 4 * nr, nr, nt, n, Np, ridx, rw, rl, res);
}

// ------------------------------------------------------------------------ Born (S6)
//
// Background (p, v) and scattered (q, u) fields stepped together:
//   u^{n+1/2} = d_v (u^{n-1/2} - dt b D+ q^n - dt db D+ p^n)
//   q^{n+1}   = d_p (q^n - dt K D-.u^{n+1/2} - dt dK D-.v^{n+1/2}) + dt dK w_n beta / dx^2
struct BornArgs {
    const float *p0, *vx0, *vz0, *q0, *ux0, *uz0;   // background and scattered state at step n
    float *p1, *vx1, *vz1, *q1, *ux1, *uz1;         // ... at step n+1
    Model mo;
    Pert pe;
    Dims d;
    Stencil st;
    Source src;
    int n, tz, nshots;
};

template <int M>
struct BornSmem {
    float pr[2 * M + BORN_WPD][WROW];
    float qr[2 * M + BORN_WPD][WROW];
    float stg[BORN_WPD + 1][10][WROW];
    float vr[2][WROW];
    float ur[2][WROW];
    float scl[BORN_WPD + 1][4];            // az(j), azh(r) of each stage
};

template <int M>
__device__ __forceinline__ void born_body(const BornArgs &a, const Strip &sp, BornSmem<M> &sh)
{
    constexpr int R = 2 * M, NS = BORN_WPD + 1, NF = 10, NP = 2 * M + BORN_WPD;
    const Dims &d = a.d;
    const Model &mo = a.mo;
    const Pert &pe = a.pe;
    const Stencil &st = a.st;
    const int n = a.n, tz = a.tz;
    float(*spr)[WROW] = sh.pr;
    float(*sqr)[WROW] = sh.qr;
    float(*stg)[NF][WROW] = sh.stg;
    float(*svr)[WROW] = sh.vr;
    float(*sur)[WROW] = sh.ur;
    const int lane = threadIdx.x & 31;
    const LaneMap L = lane_map(lane, sp.x0, d);
    for (int k = lane; k < 2 * WROW; k += 32) { (&svr[0][0])[k] = 0.f; (&sur[0][0])[k] = 0.f; }
    const long long so = (long long)sp.s * d.Np;
    const float *P0 = a.p0 + so, *VX0 = a.vx0 + so, *VZ0 = a.vz0 + so;
    const float *Q0 = a.q0 + so, *UX0 = a.ux0 + so, *UZ0 = a.uz0 + so;
    float *P1 = a.p1 + so, *VX1 = a.vx1 + so, *VZ1 = a.vz1 + so;
    float *Q1 = a.q1 + so, *UX1 = a.ux1 + so, *UZ1 = a.uz1 + so;
    const SrcCells sc = src_cells(a.src, sp.s, d.Px);
    const float wn = __ldg(a.src.wav + n);
    const float4 axv = ldg_if(mo.ax + L.mc, L.in), axhv = ldg_if(mo.axh + L.mc, L.in);
    const int z0 = sp.z0, zend = min(z0 + tz, d.Nz), f0 = z0 - R;
    const bool hsrc = strip_has_src(sc, sp.x0, z0, zend);
    // rows the strip's outputs depend on (the others stream in as zeros, reading nothing):
    // p, q rows f >= z0 - 2M + 1, v_z, u_z rows r >= z0 - M, v_x, u_x, model rows j >= z0
    auto issue = [&](int g, int ps, int ss) {
        const int f = f0 + g, r = f - M, j = f - R + 1;
        const bool vf = f >= max(0, z0 - R + 1) && f < d.Nz, vr = r >= max(0, z0 - M) && r < d.Nz,
                   vj = j >= z0 && j < d.Nz;
        float *pr = spr[ps], *qr = sqr[ps];
        float(*sg)[WROW] = stg[ss];
        const int of = f * d.Px, orr = r * d.Px, oj = j * d.Px;
        if (lane == 0) {
            cp4(&sh.scl[ss][0], mo.az, j, FWI_IN(vj, j, 1, d.Nz, mo.status));
            cp4(&sh.scl[ss][1], mo.azh, r, FWI_IN(vr, r, 1, d.Nz, mo.status));
        }
        const long long np = d.Np;
        int *stt = mo.status;
        const bool zo = FWI_IN(vr && L.in && L.own, orr + L.mc, 4, np, stt),
                   xo = FWI_IN(vj && L.in, oj + L.mc, 4, np, stt), fm = FWI_IN(vf && L.in, of + L.mc, 4, np, stt);
        cp16(pr + L.mo, P0, of + L.mc, fm);
        cp16(qr + L.mo, Q0, of + L.mc, fm);
        if (!L.own) {
            const bool fe = FWI_IN(vf && L.ein, of + L.ec, 4, np, stt);
            cp16(pr + L.eo, P0, of + L.ec, fe);
            cp16(qr + L.eo, Q0, of + L.ec, fe);
        }
        cp16(sg[0] + L.mo, VZ0, orr + L.mc, zo);
        cp16(sg[1] + L.mo, UZ0, orr + L.mc, zo);
        cp16(sg[2] + L.mo, mo.bz, orr + L.mc, zo);
        cp16(sg[3] + L.mo, pe.dbz, orr + L.mc, zo);
        cp16(sg[4] + L.mo, VX0, oj + L.mc, xo);
        cp16(sg[5] + L.mo, UX0, oj + L.mc, xo);
        cp16(sg[6] + L.mo, mo.bx, oj + L.mc, xo);
        cp16(sg[7] + L.mo, pe.dbx, oj + L.mc, xo);
        cp16(sg[8] + L.mo, mo.K, oj + L.mc, xo && L.own);
        cp16(sg[9] + L.mo, pe.dK, oj + L.mc, xo && L.own);
        cp_commit();
    };
    float4 vq[R], uq[R];   // vz and uz rows r-2M+1 .. r, oldest first
    float4 pq[R];          // this lane's own p float4 of rows g-2M+1 .. g (z-stencil from registers)
#pragma unroll
    for (int k = 0; k < R; ++k) { vq[k] = f4(0.f); uq[k] = f4(0.f); pq[k] = f4(0.f); }
#pragma unroll
    for (int g = 0; g < BORN_WPD; ++g) issue(g, g, g);
    RingPos<NP> P;      // ring position of row g
    RingPos<NS> S;      // stage of row g
    const int fend = zend + R - 1;
#pragma unroll 2   // two rows per trip: half the register-queue shifts (measured: 1 < 2 > 4)
    for (int f = f0; f < fend; ++f) {
        const int g = f - f0;
        __syncwarp();
        issue(g + BORN_WPD, P(BORN_WPD), S(BORN_WPD));
        cp_wait<BORN_WPD>();
        __syncwarp();
        float(*sg)[WROW] = stg[S(0)];
        const float az = sh.scl[S(0)][0], azh = sh.scl[S(0)][1];
        const int r = f - M;
#pragma unroll
        for (int q = 0; q < R - 1; ++q) pq[q] = pq[q + 1];
        pq[R - 1] = ld4(spr[P(0)] + L.mo);
        float4 gp = f4(0.f), gq = f4(0.f);     // -dt D+z p, -dt D+z q (pq[q] is row g - 2M + 1 + q)
#pragma unroll
        for (int k = 1; k <= M; ++k) {
            const int a = P(k - M), b = P(1 - M - k);
            gp = ptap(st.nc[k - 1], pq[M - 1 + k], pq[M - k], gp);
            gq = ptap(st.nc[k - 1], ld4(sqr[a] + L.mo), ld4(sqr[b] + L.mo), gq);
        }
        const float4 fz = pmul(azh, axv), bz = ld4(sg[2] + L.mo);
        const float4 vz = pmul(fz, pfma(bz, gp, ld4(sg[0] + L.mo)));
        const float4 uz = pmul(fz, pfma(ld4(sg[3] + L.mo), gp, pfma(bz, gq, ld4(sg[1] + L.mo))));
        if (FWI_IN(L.wr && r >= z0 && r < zend, (long long)r * d.Px + L.mc, 4, d.Np, mo.status)) {
            st4(VZ1 + r * d.Px + L.mc, vz);
            st4(UZ1 + r * d.Px + L.mc, uz);
        }
#pragma unroll
        for (int q = 0; q < R - 1; ++q) { vq[q] = vq[q + 1]; uq[q] = uq[q + 1]; }
        vq[R - 1] = vz;
        uq[R - 1] = uz;
        const int j = f - R + 1;
        const bool row = j >= z0 && j < zend;
        const int sj = P(1 - R);
        const float *prow = spr[sj], *qrow = sqr[sj];
        const float4 fx = pmul(az, axhv), bx = ld4(sg[6] + L.mo);
        const float4 gpx = row_dplus<M>(prow, L.mo, pq[0], st.nc);
        const float4 vx = pmul(fx, pfma(bx, gpx, ld4(sg[4] + L.mo)));
        const float4 ux = pmul(fx, pfma(ld4(sg[7] + L.mo), gpx, pfma(bx, row_dplus<M>(qrow, L.mo, st.nc), ld4(sg[5] + L.mo))));
        float *vrow = svr[f & 1], *urow = sur[f & 1];
        st4(vrow + L.mo, vx);
        st4(urow + L.mo, ux);
        const bool jw = FWI_IN(row && L.wr, (long long)j * d.Px + L.mc, 4, d.Np, mo.status);
        if (jw) {
            st4(VX1 + j * d.Px + L.mc, vx);
            st4(UX1 + j * d.Px + L.mc, ux);
        }
        __syncwarp();
        if (jw) {
            float4 dv = row_dminus<M>(vrow, L.mo, vx, st.nc), du = row_dminus<M>(urow, L.mo, ux, st.nc);
#pragma unroll
            for (int k = 1; k <= M; ++k) {   // vq[q] is vz row j - M + q
                dv = ptap(st.nc[k - 1], vq[M + k - 1], vq[M - k], dv);
                du = ptap(st.nc[k - 1], uq[M + k - 1], uq[M - k], du);
            }
            const float4 K = ld4(sg[8] + L.mo), dK = ld4(sg[9] + L.mo), fp = pmul(az, axv);
            float4 pn = pmul(fp, pfma(K, dv, pq[0]));
            float4 qn = pmul(fp, pfma(dK, dv, pfma(K, du, ld4(qrow + L.mo))));
            if (hsrc) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (sc.j[k] == j && sc.i[k] >= L.mc && sc.i[k] < L.mc + 4) {
                        const int c = sc.i[k] - L.mc;
                        addc(pn, c, comp(K, c) * wn * sc.w[k]);
                        addc(qn, c, comp(dK, c) * wn * sc.w[k]);
                    }
            }
            st4(P1 + j * d.Px + L.mc, pn);
            st4(Q1 + j * d.Px + L.mc, qn);
        }
        P.next();
        S.next();
    }
    cp_wait<0>();
}

template <int M, int MINB>
__global__ void __launch_bounds__(32, MINB) k_born_warp(BornArgs a, Tail tl)
{
    extern __shared__ __align__(16) unsigned char fwi_smem[];
    const int w = blockIdx.x, nw = strip_warps(a.d, a.tz, a.nshots);
    if (w >= nw) {   // a sampling warp
        sample_tail(tl, (w - nw) * 32 + (threadIdx.x & 31));
        return;
    }
    bool valid;
    const Strip sp = strip_at(w, a.d, a.tz, a.nshots, valid);
    born_body<M>(a, sp, *reinterpret_cast<BornSmem<M> *>(fwi_smem));
}

template <int M>
__global__ void __launch_bounds__(32) k_born_batch(const __grid_constant__ BatchTable<BornArgs> t)
{
    extern __shared__ __align__(16) unsigned char fwi_smem[];
    BornSmem<M> &sh = *reinterpret_cast<BornSmem<M> *>(fwi_smem);
    const int w = blockIdx.x;
    if (w >= t.wstart[t.njobs]) return;
    int local;
    const BornArgs &a = t.jobs[job_of(w, t.wstart, t.njobs, local)];
    bool valid;
    const Strip sp = strip_at(local, a.d, a.tz, a.nshots, valid);
    if (!valid) return;
    born_body<M>(a, sp, sh);
}

// dynamic shared memory of one block of each family
template <int M>
constexpr size_t fwd_smem() { return sizeof(FwdSmem<M>) * FWD_WPB; }
template <int M>
constexpr size_t adj_smem() { return sizeof(AdjSmem<M>); }
template <int M>
constexpr size_t born_smem() { return sizeof(BornSmem<M>); }
static_assert(fwd_smem<4>() <= 227 * 1024 && adj_smem<4>() <= 227 * 1024 && born_smem<4>() <= 227 * 1024,
              "staging exceeds the shared memory of a block");

static_assert(sizeof(BatchTable<FwdArgs>) + sizeof(SmallTable) <= 32000,
              "forward batch and per-receiver tables exceed the kernel parameter space");
static_assert(sizeof(BatchTable<FwdArgs>) <= 32000 && sizeof(BatchTable<AdjArgs>) <= 32000 &&
                  sizeof(BatchTable<BornArgs>) <= 32000,
              "batch table exceeds the kernel parameter space");

}  // namespace fwi
