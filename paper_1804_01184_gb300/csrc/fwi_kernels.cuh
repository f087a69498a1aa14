// fwi_kernels.cuh -- device code of libfwi.so (sm_103a).
//
// Staggered-grid finite differences of the 2-D variable-density acoustic wave equation
// (Sec. "Scheme III" of arXiv:1804.01184; the operator of eq. param_full), the Born
// linearisation of the same scheme, and the adjoint scheme with the gradient fused in.
//
// Discretisation (the paper gives none of it; the readings are documented with the API):
//   p, K on nodes (i, j); vx on (i+1/2, j); vz on (i, j+1/2); zero outside the grid.
//   D+ f at i+1/2 = (1/dx) sum_k c_k (f[i+k] - f[i-k+1]);  D- g at i = (1/dx) sum_k c_k (g[i+k-1] - g[i-k]).
//   v^{n+1/2} = d_v (v^{n-1/2} - dt b D+ p^n);  p^{n+1} = d_p (p^n - dt K D-.v^{n+1/2}) + source.
//   Sponge factors are separable: d(i, j) = a_x(i) a_z(j).
//
// Memory layout in HBM: every field is [shot][Nz][Px] float32 with the row pitch Px a
// multiple of 32 floats (128-byte rows); columns Nx..Px-1 stay zero and count as outside.
// Model arrays (K, bx, bz) are [Nz][Px], shared by all shots of a launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fwi {

struct Dims {
    int Nx, Nz, Px;       // computational grid and row pitch
    int nx, nz, S;        // physical grid and sponge width
    long long Np;         // Px * Nz: floats per field per shot
};

// c_k * dt / dx: the stencil weights with the time step and spacing folded in, and their
// negatives (a subtracted stencil term becomes one fused multiply-add)
struct Stencil {
    float c[4];
    float nc[4];
};

// status bits recorded by the kernels
enum : int { ST_EINVAL = 1, ST_ECFL = 2, ST_EBOUNDS = 8 };

// Checked builds (-DFWI_CHECKED, the debug build): every global load and store of the time-step
// kernels first tests its offset against the size of its field; a failing test sets
// ST_EBOUNDS in the operation's status word and the access is skipped (nothing traps), and
// fwi_status() reports it.  In the default build the tests compile away.
#ifdef FWI_CHECKED
__device__ __forceinline__ bool in_field(long long off, long long len, long long lim, int *status)
{
    if (off >= 0 && off + len <= lim) return true;
    if (status) atomicOr(status, ST_EBOUNDS);
    return false;
}
#define FWI_IN(valid, off, len, lim, status) ((valid) && ::fwi::in_field((off), (len), (lim), (status)))
#else
#define FWI_IN(valid, off, len, lim, status) (valid)
#endif

__device__ __forceinline__ long long cell(const Dims &d, int i, int j) { return (long long)j * d.Px + i; }

// ------------------------------------------------------------------ model build (S1)

// Contrast pair -> (K, rho) for each parameterization of Table 1 (m = m_o (1 + xi);
// K = rho vp^2, Ip = rho vp).  Returns false when a contrast leaves 1 + xi <= 0.
__device__ __forceinline__ bool kr_of(int pz, double a, double b, double vp_o, double rho_o,
                                      double &K, double &rho)
{
    if (!(a > -1.0) || !(b > -1.0)) return false;
    const double Ko = rho_o * vp_o * vp_o, Io = rho_o * vp_o;
    switch (pz) {
    case 0: { double v = vp_o * (1.0 + a); rho = rho_o * (1.0 + b); K = rho * v * v; return true; }
    case 1: { double ip = Io * (1.0 + a); rho = rho_o * (1.0 + b); K = ip * ip / rho; return true; }
    case 2: { double v = vp_o * (1.0 + a), ip = Io * (1.0 + b); rho = ip / v; K = ip * v; return true; }
    case 3: K = Ko * (1.0 + a); rho = rho_o * (1.0 + b); return true;
    case 4: K = Ko / (1.0 + a); rho = rho_o / (1.0 + b); return true;
    }
    return false;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// K, bx = 2/(rho_i + rho_{i+1}), bz likewise, on the padded grid (padding copies the
// nearest physical cell; the last node reuses its own rho).  Checks 1 + xi > 0 and the
// CFL bound dt vp sqrt(2) sum|c_k| / dx <= 1.
__global__ void k_model(const float *__restrict__ xa, const float *__restrict__ xb, int pz,
                        double vp_o, double rho_o, double cfl_coef, Dims d,
                        float *__restrict__ K, float *__restrict__ bx, float *__restrict__ bz,
                        int *status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= d.Px || j >= d.Nz) return;
    const long long o = cell(d, i, j);
    if (i >= d.Nx) { K[o] = 0.f; bx[o] = 0.f; bz[o] = 0.f; return; }
    auto phys = [&](int ii, int jj, double &Kv, double &rv) {
        int pi = clampi(ii - d.S, 0, d.nx - 1), pj = clampi(jj - d.S, 0, d.nz - 1);
        long long q = (long long)pj * d.nx + pi;
        return kr_of(pz, xa[q], xb[q], vp_o, rho_o, Kv, rv);
    };
    double Kc, rc, Kx, rx, Kz, rz;
    bool ok = phys(i, j, Kc, rc);
    ok = phys(i + 1 < d.Nx ? i + 1 : i, j, Kx, rx) && ok;
    ok = phys(i, j + 1 < d.Nz ? j + 1 : j, Kz, rz) && ok;
    if (!ok) { atomicOr(status, ST_EINVAL); K[o] = 0.f; bx[o] = 0.f; bz[o] = 0.f; return; }
    if (sqrt(Kc / rc) * cfl_coef > 1.0) atomicOr(status, ST_ECFL);
    K[o] = (float)Kc;
    bx[o] = (float)(2.0 / (rc + rx));
    bz[o] = (float)(2.0 / (rc + rz));
}

// Born perturbation of the model: dK = J dxi, drho likewise (Jacobian of the map above),
// dbx = -bx^2/2 (drho_i + drho_{i+1}), dbz likewise.
__device__ __forceinline__ void jac_of(int pz, double a, double b, double vp_o, double rho_o,
                                       double &dKa, double &dKb, double &dra, double &drb)
{
    const double Ko = rho_o * vp_o * vp_o, Io = rho_o * vp_o;
    switch (pz) {
    case 0: { double v = vp_o * (1.0 + a), r = rho_o * (1.0 + b);
              dKa = 2.0 * r * v * vp_o; dKb = rho_o * v * v; dra = 0.0; drb = rho_o; break; }
    case 1: { double ip = Io * (1.0 + a), r = rho_o * (1.0 + b);
              dKa = 2.0 * ip * Io / r; dKb = -ip * ip * rho_o / (r * r); dra = 0.0; drb = rho_o; break; }
    case 2: { double v = vp_o * (1.0 + a), ip = Io * (1.0 + b);
              dKa = ip * vp_o; dKb = Io * v; dra = -ip * vp_o / (v * v); drb = Io / v; break; }
    case 3: dKa = Ko; dKb = 0.0; dra = 0.0; drb = rho_o; break;
    default: dKa = -Ko / ((1.0 + a) * (1.0 + a)); dKb = 0.0; dra = 0.0;
             drb = -rho_o / ((1.0 + b) * (1.0 + b)); break;
    }
}

__global__ void k_model_pert(const float *__restrict__ xa, const float *__restrict__ xb,
                             const float *__restrict__ da, const float *__restrict__ db, int pz,
                             double vp_o, double rho_o, Dims d, float *__restrict__ dK,
                             float *__restrict__ dbx, float *__restrict__ dbz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= d.Px || j >= d.Nz) return;
    const long long o = cell(d, i, j);
    if (i >= d.Nx) { dK[o] = 0.f; dbx[o] = 0.f; dbz[o] = 0.f; return; }
    auto pert = [&](int ii, int jj, double &dKv, double &drv, double &rv) {
        int pi = clampi(ii - d.S, 0, d.nx - 1), pj = clampi(jj - d.S, 0, d.nz - 1);
        long long q = (long long)pj * d.nx + pi;
        double a = xa[q], b = xb[q], Kv, j0, j1, j2, j3;
        kr_of(pz, a, b, vp_o, rho_o, Kv, rv);
        jac_of(pz, a, b, vp_o, rho_o, j0, j1, j2, j3);
        dKv = j0 * da[q] + j1 * db[q];
        drv = j2 * da[q] + j3 * db[q];
    };
    double dKc, drc, rc, t, drx, rx, drz, rz;
    pert(i, j, dKc, drc, rc);
    pert(i + 1 < d.Nx ? i + 1 : i, j, t, drx, rx);
    pert(i, j + 1 < d.Nz ? j + 1 : j, t, drz, rz);
    const double bxv = 2.0 / (rc + rx), bzv = 2.0 / (rc + rz);
    dK[o] = (float)dKc;
    dbx[o] = (float)(-0.5 * bxv * bxv * (drc + drx));
    dbz[o] = (float)(-0.5 * bzv * bzv * (drc + drz));
}

// Sponge profile along one axis: n physical nodes, S cells each side; half = 1 for the
// half nodes.  sigma = sigma_max (delta/S)^2, sigma_max = 3 v ln(1/R) / (2 S dx), d = exp(-sigma dt).
__global__ void k_sponge(float *__restrict__ out, int len, int n, int S, double dx, double dt,
                         double v, double R, int half)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    const int N = n + 2 * S;
    if (i >= N) { out[i] = 0.f; return; }
    const double u = i + (half ? 0.5 : 0.0);
    double delta = 0.0;
    if (u < S) delta = S - u;
    if (u > S + n - 1) delta = u - (S + n - 1);
    if (S == 0 || delta == 0.0) { out[i] = 1.f; return; }
    const double smax = 3.0 * v * log(1.0 / R) / (2.0 * S * dx);
    const double q = delta / S;
    out[i] = (float)exp(-smax * q * q * dt);
}

// Bilinear footprint of point k: four (cell offset, weight * scale) pairs.  A point on the
// last node puts its weight on (i0 + 1).  Points outside the physical grid flag EINVAL.
__global__ void k_geometry(const float *__restrict__ xy, int n, Dims d, double dx, double scale,
                           long long *__restrict__ idx, float *__restrict__ w, int *status)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double x = xy[2 * k], z = xy[2 * k + 1];
    if (!(x >= 0.0 && z >= 0.0 && x <= (d.nx - 1) * dx && z <= (d.nz - 1) * dx)) {
        atomicOr(status, ST_EINVAL);
        for (int c = 0; c < 4; ++c) { idx[4 * k + c] = 0; w[4 * k + c] = 0.f; }
        return;
    }
    const double fx = x / dx + d.S, fz = z / dx + d.S;
    int i0 = (int)floor(fx), j0 = (int)floor(fz);
    if (i0 > d.Nx - 2) i0 = d.Nx - 2;
    if (j0 > d.Nz - 2) j0 = d.Nz - 2;
    const double tx = fx - i0, tz = fz - j0;
    idx[4 * k + 0] = cell(d, i0, j0);          w[4 * k + 0] = (float)(scale * (1.0 - tx) * (1.0 - tz));
    idx[4 * k + 1] = cell(d, i0 + 1, j0);      w[4 * k + 1] = (float)(scale * tx * (1.0 - tz));
    idx[4 * k + 2] = cell(d, i0, j0 + 1);      w[4 * k + 2] = (float)(scale * (1.0 - tx) * tz);
    idx[4 * k + 3] = cell(d, i0 + 1, j0 + 1);  w[4 * k + 3] = (float)(scale * tx * tz);
}

// Receiver footprints that share a cell, chained for a deterministic adjoint injection:
// entry k (receiver k/4, corner k%4) gets the next entry with the same cell (n4 if none) in
// bits 0..29, and bit 30 set when no earlier entry has its cell.  O(n4^2), run once.
constexpr int CHAIN_FIRST = 1 << 30;

__global__ void k_receiver_chain(const long long *__restrict__ idx, int n4, int *__restrict__ rl)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n4) return;
    const long long c = idx[k];
    bool first = true;
    for (int m = 0; m < k && first; ++m) first = idx[m] != c;
    int nx = n4;
    for (int m = k + 1; m < n4; ++m)
        if (idx[m] == c) { nx = m; break; }
    rl[k] = nx | (first ? CHAIN_FIRST : 0);
}

// ------------------------------------------------------------ shared kernel arguments

struct Model {
    const float *K, *bx, *bz, *ax, *axh, *az, *azh;
    int *status;            // the operation's status word (checked builds record out-of-range accesses)
};

struct Source {
    const long long *idx;   // [shot][4] cell offsets (relative to the shot's field)
    const float *w;         // [shot][4] dt beta / dx^2
    const float *wav;       // wavelet, sample n at (n+1/2) dt
};

// Born perturbation of the model: dK, dbx, dbz on the padded grid
struct Pert {
    const float *dK, *dbx, *dbz;
};

// trace[s][r][n] = sum_c beta_rc p^{n+1}[cell_rc]
__global__ void k_sample(const float *__restrict__ p, int ns, int nr, int nt, int n, long long Np,
                         const long long *__restrict__ ridx, const float *__restrict__ rw,
                         float *__restrict__ traces)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns * nr) return;
    const int s = t / nr, r = t - s * nr;
    const float *ps = p + (long long)s * Np;
    float v = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (FWI_IN(true, ridx[4 * r + c], 1, Np, nullptr)) v += rw[4 * r + c] * ps[ridx[4 * r + c]];
    traces[(long long)t * nt + n] = v;
}

// --------------------------------------------------------------- adjoint + gradient (S7)

// ------------------------------------------------------------------ reductions (S5, S8)

constexpr int RED_THREADS = 256;

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[RED_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        v = l < RED_THREADS / 32 ? sh[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// r = traces - data (in place in `tr`), partial[blockIdx.x] = 1/2 sum r^2 (FP64).
// J = 1/2 sum w (tr - data)^2 in FP64 by one block (a fixed summation order, no scratch): the
// least-squares misfit of one set of traces (Sec. "Modelling and Inversion"), each trace
// (nt samples) weighted by w[trace] (w null: 1).
__global__ void __launch_bounds__(RED_THREADS) k_misfit(const float *__restrict__ tr, const float *__restrict__ data,
                                                       long long n, const float *__restrict__ w, int nt,
                                                       double *__restrict__ out)
{
    double acc = 0.0;
    for (long long k = threadIdx.x; k < n; k += RED_THREADS) {
        const double r = (double)tr[k] - (double)data[k];
        acc += w ? 0.5 * (double)w[k / nt] * r * r : 0.5 * r * r;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) *out = acc;
}

// Residual in place, tr <- w (tr - data), and per-block partial misfits 1/2 w (tr - data)^2:
// the adjoint source of J = 1/2 sum w r^2 (w null: 1; w per trace of nt samples).
__global__ void __launch_bounds__(RED_THREADS) k_residual(float *__restrict__ tr, const float *__restrict__ data,
                                                          long long n, double *__restrict__ partial,
                                                          const float *__restrict__ w, int nt)
{
    double acc = 0.0;
    for (long long k = (long long)blockIdx.x * RED_THREADS + threadIdx.x; k < n;
         k += (long long)gridDim.x * RED_THREADS) {
        const float r = tr[k] - data[k];
        if (w) {
            const float wk = w[k / nt];
            tr[k] = wk * r;
            acc += 0.5 * (double)wk * (double)r * (double)r;
        } else {
            tr[k] = r;
            acc += 0.5 * (double)r * (double)r;
        }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// out[0] = sum of partial[0..n) in a fixed order (single block).
__global__ void __launch_bounds__(RED_THREADS) k_sum_final(const double *__restrict__ partial, int n,
                                                           double *__restrict__ out)
{
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += RED_THREADS) acc += partial[k];
    acc = block_sum(acc);
    if (threadIdx.x == 0) out[0] = acc;
}

// Knuth's TwoSum: s + v rounded, with the exact rounding error added to c (no FMA contraction:
// every operation is an explicitly rounded add).  A run of these keeps the sum of FP32 values
// as the unevaluated pair s + c, exact to about twice FP32 precision.
__device__ __forceinline__ void two_sum(float &s, float &c, float v)
{
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    s = t;
    c = __fadd_rn(c, e);
}

// Gradient accumulation in time: every adjoint launch adds one step's zero-lag products to
// FP32 per-shot-slot fields (one red per address per launch, so the order is fixed); after a
// chunk of steps the slots are flushed into FP64 running sums over shots (and then cleared by
// the host with a memset).  A block of FLUSH_X x FLUSH_Y threads takes FLUSH_X float4 of cells
// of field blockIdx.y (Np is a multiple of 32): thread (x, y) sums slots y, y + FLUSH_Y, ... with
// TwoSum, the FLUSH_Y partial pairs are combined in y order -- a fixed order for a given slot
// count -- and the pair is added to the FP64 running sum.  (The FP64 units of this GPU are few:
// widening every slot value would make the flush FP64-bound; the compensated FP32 sum needs
// four FP64 operations a cell.)
constexpr int FLUSH_X = 32, FLUSH_Y = 8, FLUSH_UNROLL = 4;

__global__ void __launch_bounds__(FLUSH_X * FLUSH_Y) k_acc_flush(const float *__restrict__ accK,
                                                                 const float *__restrict__ accBx,
                                                                 const float *__restrict__ accBz, int nslots, long long Np,
                                                                 double *__restrict__ sK, double *__restrict__ sX,
                                                                 double *__restrict__ sZ)
{
    __shared__ float ps[FLUSH_Y][FLUSH_X][4], pc[FLUSH_Y][FLUSH_X][4];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const long long e = ((long long)blockIdx.x * FLUSH_X + tx) * 4;
    const float *__restrict__ acc = blockIdx.y == 0 ? accK : blockIdx.y == 1 ? accBx : accBz;
    double *__restrict__ sum = blockIdx.y == 0 ? sK : blockIdx.y == 1 ? sX : sZ;
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    if (e < Np)
        for (int s0 = ty; s0 < nslots; s0 += FLUSH_Y * FLUSH_UNROLL) {
            float4 v[FLUSH_UNROLL];
#pragma unroll
            for (int u = 0; u < FLUSH_UNROLL; ++u) {   // independent loads first
                const int sl = s0 + u * FLUSH_Y;
                v[u] = sl < nslots ? __ldcs(reinterpret_cast<const float4 *>(acc + sl * Np + e))
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < FLUSH_UNROLL; ++u)
                if (s0 + u * FLUSH_Y < nslots) {
                    two_sum(s[0], c[0], v[u].x);
                    two_sum(s[1], c[1], v[u].y);
                    two_sum(s[2], c[2], v[u].z);
                    two_sum(s[3], c[3], v[u].w);
                }
        }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ps[ty][tx][k] = s[k];
        pc[ty][tx][k] = c[k];
    }
    __syncthreads();
    if (ty == 0 && e < Np) {
        float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int y = 0; y < FLUSH_Y; ++y)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                two_sum(S[k], C[k], ps[y][tx][k]);
                C[k] = __fadd_rn(C[k], pc[y][tx][k]);
            }
        double2 *o = reinterpret_cast<double2 *>(sum + e);
        const double2 lo = o[0], hi = o[1];
        o[0] = make_double2(lo.x + ((double)S[0] + (double)C[0]), lo.y + ((double)S[1] + (double)C[1]));
        o[1] = make_double2(hi.x + ((double)S[2] + (double)C[2]), hi.y + ((double)S[3] + (double)C[3]));
    }
}

// Per padded cell, FP64, in place on the running sums of k_acc_flush:
// gK = sum accK / K;  hx = g_bx * d bx/d rho_each = (sum accBx) bx^2/2 (g_bx = -sum accBx,
// d bx / d rho = -bx^2/2 for each of its two cells), hz likewise.
__global__ void k_grad_cells(const float *__restrict__ K, const float *__restrict__ bx,
                             const float *__restrict__ bz, Dims d, double *__restrict__ gK,
                             double *__restrict__ hx, double *__restrict__ hz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= d.Nx || j >= d.Nz) return;
    const long long m = cell(d, i, j);
    const double b1 = bx[m], b2 = bz[m];
    gK[m] = gK[m] / (double)K[m];
    hx[m] = 0.5 * b1 * b1 * hx[m];
    hz[m] = 0.5 * b2 * b2 * hz[m];
}

// Per physical cell: fold the padding it feeds, form g_rho from the buoyancy nodes that
// touch each padded cell, then the chain rule of every parameterization at the cell's
// (K, rho) (closed-form Jacobians of the maps of Table 1), written as grads[5][2][nz][nx].
__global__ void k_grad_final(const double *__restrict__ gK, const double *__restrict__ hx,
                             const double *__restrict__ hz, const float *__restrict__ xa,
                             const float *__restrict__ xb, int pz, double vp_o, double rho_o, Dims d,
                             double *__restrict__ grads)
{
    const int pi = blockIdx.x * blockDim.x + threadIdx.x, pj = blockIdx.y * blockDim.y + threadIdx.y;
    if (pi >= d.nx || pj >= d.nz) return;
    const int ilo = pi == 0 ? 0 : pi + d.S, ihi = pi == d.nx - 1 ? d.Nx - 1 : pi + d.S;
    const int jlo = pj == 0 ? 0 : pj + d.S, jhi = pj == d.nz - 1 ? d.Nz - 1 : pj + d.S;
    double sK = 0.0, sR = 0.0;
    for (int j = jlo; j <= jhi; ++j)
        for (int i = ilo; i <= ihi; ++i) {
            const long long m = cell(d, i, j);
            sK += gK[m];
            double gr = hx[m] + hz[m];                       // buoyancy nodes at i+1/2, j+1/2
            if (i > 0) gr += hx[m - 1];                      // node at i-1/2
            if (i == d.Nx - 1) gr += hx[m];                  // last node reuses rho_i twice
            if (j > 0) gr += hz[m - d.Px];
            if (j == d.Nz - 1) gr += hz[m];
            sR += gr;
        }
    const long long q = (long long)pj * d.nx + pi;
    double K, rho;
    kr_of(pz, xa[q], xb[q], vp_o, rho_o, K, rho);
    const double vp = sqrt(K / rho), Ko = rho_o * vp_o * vp_o, Io = rho_o * vp_o;
    const long long P = (long long)d.nx * d.nz;
    // (A) vp-rho: K = rho vp^2
    grads[0 * P + q] = vp_o * 2.0 * rho * vp * sK;
    grads[1 * P + q] = rho_o * (sR + vp * vp * sK);
    // (B) Ip-rho: K = Ip^2 / rho
    grads[2 * P + q] = Io * 2.0 * vp * sK;
    grads[3 * P + q] = rho_o * (sR - vp * vp * sK);
    // (C) vp-Ip: rho = Ip/vp, K = Ip vp
    grads[4 * P + q] = vp_o * (rho * vp * sK - rho / vp * sR);
    grads[5 * P + q] = Io * (vp * sK + sR / vp);
    // (D) K-rho
    grads[6 * P + q] = Ko * sK;
    grads[7 * P + q] = rho_o * sR;
    // (E) 1/K-1/rho: K = K_o/(1+a), rho = rho_o/(1+b)
    grads[8 * P + q] = -K * K / Ko * sK;
    grads[9 * P + q] = -rho * rho / rho_o * sR;
}

}  // namespace fwi
