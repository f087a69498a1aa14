/*
 * fwi_oracle.c -- plain FP64 CPU oracle for the Scheme III hot path of
 *   M. Bharadwaj, W. Mulder, G. Drijkoningen, "A parameterization analysis for
 *   acoustic full-waveform inversion of sub-wavelength anomalies" (arXiv:1804.01184).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
 * that the CUDA path is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark load it; the library never does.  It shares
 * no source with the CUDA path.
 *
 * What it computes (every piece cites the passage of the paper it follows; where
 * the paper is silent the adopted reading is named):
 *   - contrasts -> physical model (bulk modulus K, density rho):  Sec. "Parameterization
 *     Choices", the contrast definition m_a = m_ao (1 + xi_a) and Table 1 (the five
 *     parameter pairs); Table 2 fixes the exact (non-linear) relations between them;
 *   - time-domain staggered-grid finite differences of the variable-density acoustic
 *     wave equation (the operator of eq. param_full), for forward and adjoint
 *     wavefields, absorbing boundaries on all sides:  Sec. "Scheme III";
 *   - least-squares misfit J = 1/2 sum |p - q|^2:  Sec. "Modelling and Inversion";
 *   - gradient w.r.t. the model by adjoint modelling, then the chain rule to each
 *     parameterization:  Sec. "Modelling and Inversion" (paragraph after the misfit);
 *   - Born (linearised) modelling, here the exact linearisation of the same discrete
 *     scheme (the Born idea of eq. param_born applied to Scheme III's discretisation).
 *
 * Discretisation readings (the paper gives none of these details):
 *   grid   : p, K, rho on integer nodes (i, j); vx on (i+1/2, j); vz on (i, j+1/2);
 *            arrays [Nz][Nx], x fastest; every value outside the array is zero.
 *   stencil: Taylor staggered coefficients of order 4 or 8.
 *   rho    : buoyancy on staggered nodes bx = 2/(rho_i + rho_{i+1}) (last node reuses rho).
 *   sponge : multiplicative damping d = exp(-sigma dt), sigma = sigma_max (delta/L)^2,
 *            sigma_max = 3 v ln(1/R) / (2 L), separable in x and z.
 *   source : volume injection into p, scaled by local K, bilinear weights / dx^2,
 *            wavelet sample n taken at time (n+1/2) dt (supplied by the caller).
 *   traces : bilinear sample of p^{n+1} (time (n+1) dt) at each receiver.
 *   model  : the padding cells copy the nearest physical cell.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off [-fopenmp] fwi_oracle.c -lm
 * OpenMP only splits the rows of each stencil sweep; every cell's arithmetic is the same
 * with or without it, and every reduction runs in a fixed sequential order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, nz;      /* physical nodes in x and z                                */
    int sponge;      /* padding cells added on every side (absorbing layer)      */
    int order;       /* spatial order: 4 or 8                                    */
    int nt;          /* time steps                                               */
    double dx, dt;   /* grid spacing [m] (dz = dx) and time step [s]             */
    double vp_o, rho_o;      /* reference medium (homogeneous)                   */
    double sponge_v, sponge_R; /* velocity and target reflection of the sponge   */
} og_grid;

enum { PZ_VP_RHO = 0, PZ_IP_RHO = 1, PZ_VP_IP = 2, PZ_K_RHO = 3, PZ_INVK_INVRHO = 4 };

/* ------------------------------------------------------------------ stencil */

/* Staggered first-derivative coefficients c_1..c_M (Taylor, order 2M). */
int oracle_coefficients(int order, double *c)
{
    if (order == 4) {
        c[0] = 9.0 / 8.0;
        c[1] = -1.0 / 24.0;
        return 2;
    }
    if (order == 8) {
        c[0] = 1225.0 / 1024.0;
        c[1] = -245.0 / 3072.0;
        c[2] = 49.0 / 5120.0;
        c[3] = -5.0 / 7168.0;
        return 4;
    }
    return -1;
}

static double at(const double *f, int Nx, int Nz, int i, int j)
{
    if (i < 0 || i >= Nx || j < 0 || j >= Nz) return 0.0;
    return f[(size_t)j * Nx + i];
}

/* D+ : derivative of a node field evaluated at the half node (i+1/2) (x) or (j+1/2) (z). */
static double dplus(const double *f, int Nx, int Nz, int i, int j, int axis,
                    const double *c, int M, double dx)
{
    double s = 0.0;
    for (int k = 1; k <= M; ++k) {
        if (axis == 0) s += c[k - 1] * (at(f, Nx, Nz, i + k, j) - at(f, Nx, Nz, i - k + 1, j));
        else           s += c[k - 1] * (at(f, Nx, Nz, i, j + k) - at(f, Nx, Nz, i, j - k + 1));
    }
    return s / dx;
}

/* D- : derivative of a half-node field evaluated at the node i (x) or j (z). */
static double dminus(const double *f, int Nx, int Nz, int i, int j, int axis,
                     const double *c, int M, double dx)
{
    double s = 0.0;
    for (int k = 1; k <= M; ++k) {
        if (axis == 0) s += c[k - 1] * (at(f, Nx, Nz, i + k - 1, j) - at(f, Nx, Nz, i - k, j));
        else           s += c[k - 1] * (at(f, Nx, Nz, i, j + k - 1) - at(f, Nx, Nz, i, j - k));
    }
    return s / dx;
}

/* 1-D helper for the stencil pins: out = D+ f (minus == 0) or D- f (minus == 1). */
int oracle_apply_d(int n, const double *f, double *out, int order, int minus, double dx)
{
    double c[4];
    int M = oracle_coefficients(order, c);
    if (M < 0) return -1;
    for (int i = 0; i < n; ++i)
        out[i] = minus ? dminus(f, n, 1, i, 0, 0, c, M, dx) : dplus(f, n, 1, i, 0, 0, c, M, dx);
    return 0;
}

/* ------------------------------------------------------- parameterization */

/* Contrast pair (a, b) in parameterization pz -> (K, rho).  Table 1 gives the pairs,
 * the contrast definition m = m_o (1 + xi) and K = rho vp^2, Ip = rho vp. */
int oracle_forward_map(int pz, double a, double b, double vp_o, double rho_o,
                       double *K, double *rho)
{
    const double Ip_o = rho_o * vp_o, K_o = rho_o * vp_o * vp_o;
    if (!(1.0 + a > 0.0) || !(1.0 + b > 0.0)) return -1;
    switch (pz) {
    case PZ_VP_RHO: {
        double vp = vp_o * (1.0 + a);
        *rho = rho_o * (1.0 + b);
        *K = *rho * vp * vp;
        return 0;
    }
    case PZ_IP_RHO: {
        double Ip = Ip_o * (1.0 + a);
        *rho = rho_o * (1.0 + b);
        *K = Ip * Ip / *rho;
        return 0;
    }
    case PZ_VP_IP: {
        double vp = vp_o * (1.0 + a);
        double Ip = Ip_o * (1.0 + b);
        *rho = Ip / vp;
        *K = Ip * vp;
        return 0;
    }
    case PZ_K_RHO:
        *K = K_o * (1.0 + a);
        *rho = rho_o * (1.0 + b);
        return 0;
    case PZ_INVK_INVRHO:            /* 1/K = (1/K_o)(1 + a), 1/rho = (1/rho_o)(1 + b) */
        *K = K_o / (1.0 + a);
        *rho = rho_o / (1.0 + b);
        return 0;
    }
    return -1;
}

/* Jacobian d(K, rho)/d(a, b) of oracle_forward_map at (a, b):
 * jac = [dK/da, dK/db, drho/da, drho/db].  Written from the maps above. */
static int jacobian(int pz, double a, double b, double vp_o, double rho_o, double *jac)
{
    const double Ip_o = rho_o * vp_o, K_o = rho_o * vp_o * vp_o;
    double K, rho;
    if (oracle_forward_map(pz, a, b, vp_o, rho_o, &K, &rho)) return -1;
    switch (pz) {
    case PZ_VP_RHO: {
        double vp = vp_o * (1.0 + a);
        jac[0] = 2.0 * rho * vp * vp_o;  jac[1] = rho_o * vp * vp;
        jac[2] = 0.0;                    jac[3] = rho_o;
        return 0;
    }
    case PZ_IP_RHO: {
        double Ip = Ip_o * (1.0 + a);
        jac[0] = 2.0 * Ip * Ip_o / rho;  jac[1] = -Ip * Ip / (rho * rho) * rho_o;
        jac[2] = 0.0;                    jac[3] = rho_o;
        return 0;
    }
    case PZ_VP_IP: {
        double vp = vp_o * (1.0 + a), Ip = Ip_o * (1.0 + b);
        jac[0] = Ip * vp_o;              jac[1] = Ip_o * vp;
        jac[2] = -Ip / (vp * vp) * vp_o; jac[3] = Ip_o / vp;
        return 0;
    }
    case PZ_K_RHO:
        jac[0] = K_o;  jac[1] = 0.0;
        jac[2] = 0.0;  jac[3] = rho_o;
        return 0;
    case PZ_INVK_INVRHO:
        jac[0] = -K_o / ((1.0 + a) * (1.0 + a));  jac[1] = 0.0;
        jac[2] = 0.0;  jac[3] = -rho_o / ((1.0 + b) * (1.0 + b));
        return 0;
    }
    return -1;
}

/* The five parameterizations' contrasts of one physical model (K, rho), i.e. the inverse
 * maps; used to evaluate every chain rule at the same physical point. */
static void inverse_maps(double K, double rho, double vp_o, double rho_o, double ab[5][2])
{
    const double Ip_o = rho_o * vp_o, K_o = rho_o * vp_o * vp_o;
    double vp = sqrt(K / rho), Ip = rho * vp;
    ab[PZ_VP_RHO][0] = vp / vp_o - 1.0;      ab[PZ_VP_RHO][1] = rho / rho_o - 1.0;
    ab[PZ_IP_RHO][0] = Ip / Ip_o - 1.0;      ab[PZ_IP_RHO][1] = rho / rho_o - 1.0;
    ab[PZ_VP_IP][0] = vp / vp_o - 1.0;       ab[PZ_VP_IP][1] = Ip / Ip_o - 1.0;
    ab[PZ_K_RHO][0] = K / K_o - 1.0;         ab[PZ_K_RHO][1] = rho / rho_o - 1.0;
    ab[PZ_INVK_INVRHO][0] = K_o / K - 1.0;   ab[PZ_INVK_INVRHO][1] = rho_o / rho - 1.0;
}

/* Chain rule (Sec. "Modelling and Inversion": gradient w.r.t. the base pair, then the chain
 * rule): for every physical cell, g_(a,b) = J^T (g_K, g_rho) for all five parameterizations,
 * J evaluated at the cell's (K, rho).  grads is [5][2][n]. */
int oracle_chain_rule(double vp_o, double rho_o, int n, const double *K, const double *rho,
                      const double *gK, const double *grho, double *grads)
{
    for (int c = 0; c < n; ++c) {
        double ab[5][2], jac[4];
        inverse_maps(K[c], rho[c], vp_o, rho_o, ab);
        for (int pz = 0; pz < 5; ++pz) {
            if (jacobian(pz, ab[pz][0], ab[pz][1], vp_o, rho_o, jac)) return -1;
            grads[((size_t)pz * 2 + 0) * n + c] = jac[0] * gK[c] + jac[2] * grho[c];
            grads[((size_t)pz * 2 + 1) * n + c] = jac[1] * gK[c] + jac[3] * grho[c];
        }
    }
    return 0;
}

/* -------------------------------------------------------------- model build */

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Contrasts on the physical grid -> K, rho on the padded grid (padding copies the nearest
 * physical cell) and buoyancies on the staggered nodes. */
int oracle_model_build(const og_grid *g, int pz, const double *xi_a, const double *xi_b,
                       double *K, double *rho, double *bx, double *bz)
{
    const int S = g->sponge, Nx = g->nx + 2 * S, Nz = g->nz + 2 * S;
    for (int j = 0; j < Nz; ++j)
        for (int i = 0; i < Nx; ++i) {
            int pi = clampi(i - S, 0, g->nx - 1), pj = clampi(j - S, 0, g->nz - 1);
            size_t q = (size_t)pj * g->nx + pi, o = (size_t)j * Nx + i;
            if (oracle_forward_map(pz, xi_a[q], xi_b[q], g->vp_o, g->rho_o, &K[o], &rho[o]))
                return -1;
        }
    for (int j = 0; j < Nz; ++j)
        for (int i = 0; i < Nx; ++i) {
            size_t o = (size_t)j * Nx + i;
            int ir = i + 1 < Nx ? i + 1 : i, jr = j + 1 < Nz ? j + 1 : j;
            bx[o] = 2.0 / (rho[o] + rho[(size_t)j * Nx + ir]);
            bz[o] = 2.0 / (rho[o] + rho[(size_t)jr * Nx + i]);
        }
    return 0;
}

/* ------------------------------------------------------------------ sponge */

/* Damping factors along one axis with n physical nodes and S padding cells.  half = 0: nodes
 * at integer positions u = i; half = 1: nodes at u = i + 1/2.  delta = distance (cells) into
 * the layer; sigma = sigma_max (delta / S)^2; sigma_max = 3 v ln(1/R) / (2 S dx). */
void oracle_sponge_profile(int n, int S, double dx, double dt, double v, double R, int half,
                           double *d)
{
    const int N = n + 2 * S;
    for (int i = 0; i < N; ++i) {
        double u = i + (half ? 0.5 : 0.0), delta = 0.0;
        if (u < S) delta = S - u;
        if (u > S + n - 1) delta = u - (S + n - 1);
        if (S == 0 || delta == 0.0) { d[i] = 1.0; continue; }
        double sigma_max = 3.0 * v * log(1.0 / R) / (2.0 * S * dx);
        double sigma = sigma_max * (delta / S) * (delta / S);
        d[i] = exp(-sigma * dt);
    }
}

/* ------------------------------------------------------- source / receiver */

/* Bilinear weights of a point (x, z) [m, physical origin at physical node (0,0)] on the
 * padded grid: cells (i0,j0), (i0+1,j0), (i0,j0+1), (i0+1,j0+1). */
int oracle_weights(const og_grid *g, double x, double z, long *idx, double *w)
{
    const int S = g->sponge, Nx = g->nx + 2 * S, Nz = g->nz + 2 * S;
    if (!(x >= 0.0 && z >= 0.0 && x <= (g->nx - 1) * g->dx && z <= (g->nz - 1) * g->dx))
        return -1;
    if (Nx < 2 || Nz < 2) return -1;
    double fx = x / g->dx + S, fz = z / g->dx + S;
    int i0 = (int)floor(fx), j0 = (int)floor(fz);
    if (i0 > Nx - 2) i0 = Nx - 2;   /* a point on the last node: weight 1 on (i0+1) */
    if (j0 > Nz - 2) j0 = Nz - 2;
    double tx = fx - i0, tz = fz - j0;
    idx[0] = (long)j0 * Nx + i0;        w[0] = (1.0 - tx) * (1.0 - tz);
    idx[1] = (long)j0 * Nx + i0 + 1;    w[1] = tx * (1.0 - tz);
    idx[2] = (long)(j0 + 1) * Nx + i0;  w[2] = (1.0 - tx) * tz;
    idx[3] = (long)(j0 + 1) * Nx + i0 + 1; w[3] = tx * tz;
    return 0;
}

/* ----------------------------------------------------------- common set-up */

typedef struct {
    int S, Nx, Nz, M;
    size_t N;
    double c[4];
    double *K, *rho, *bx, *bz;
    double *ax, *axh, *az, *azh;   /* separable damping: node / half-node profiles */
} model_t;

static void model_free(model_t *m)
{
    free(m->K); free(m->rho); free(m->bx); free(m->bz);
    free(m->ax); free(m->axh); free(m->az); free(m->azh);
}

static int model_init(const og_grid *g, int pz, const double *xi_a, const double *xi_b,
                      model_t *m)
{
    memset(m, 0, sizeof(*m));
    m->S = g->sponge;
    m->Nx = g->nx + 2 * m->S;
    m->Nz = g->nz + 2 * m->S;
    m->N = (size_t)m->Nx * m->Nz;
    m->M = oracle_coefficients(g->order, m->c);
    if (m->M < 0 || g->nx < 1 || g->nz < 1 || g->nt < 0) return -1;
    m->K = malloc(m->N * sizeof(double));
    m->rho = malloc(m->N * sizeof(double));
    m->bx = malloc(m->N * sizeof(double));
    m->bz = malloc(m->N * sizeof(double));
    m->ax = malloc(m->Nx * sizeof(double));
    m->axh = malloc(m->Nx * sizeof(double));
    m->az = malloc(m->Nz * sizeof(double));
    m->azh = malloc(m->Nz * sizeof(double));
    if (oracle_model_build(g, pz, xi_a, xi_b, m->K, m->rho, m->bx, m->bz)) {
        model_free(m);
        return -1;
    }
    oracle_sponge_profile(g->nx, m->S, g->dx, g->dt, g->sponge_v, g->sponge_R, 0, m->ax);
    oracle_sponge_profile(g->nx, m->S, g->dx, g->dt, g->sponge_v, g->sponge_R, 1, m->axh);
    oracle_sponge_profile(g->nz, m->S, g->dx, g->dt, g->sponge_v, g->sponge_R, 0, m->az);
    oracle_sponge_profile(g->nz, m->S, g->dx, g->dt, g->sponge_v, g->sponge_R, 1, m->azh);
    return 0;
}

/* damping factors of the three node types at cell (i, j) */
#define DP(m, i, j)  ((m)->ax[i] * (m)->az[j])
#define DVX(m, i, j) ((m)->axh[i] * (m)->az[j])
#define DVZ(m, i, j) ((m)->ax[i] * (m)->azh[j])

/* One forward time step n (Sec. Scheme III; the discretisation readings above):
 *   v^{n+1/2} = d_v (v^{n-1/2} - dt b D+ p^n)
 *   p^{n+1}   = d_p (p^n - dt K (Dx- vx + Dz- vz)) + dt K_c w_n beta_c / dx^2  at source cells
 * divv (optional) receives Dx- vx^{n+1/2} + Dz- vz^{n+1/2}. */
static void step_forward(const og_grid *g, const model_t *m, double *p, double *vx, double *vz,
                         const long *sidx, const double *sw, double wn, double *divv)
{
    const int Nx = m->Nx, Nz = m->Nz, M = m->M;
    const double dt = g->dt, dx = g->dx;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < Nz; ++j)
        for (int i = 0; i < Nx; ++i) {
            size_t o = (size_t)j * Nx + i;
            vx[o] = DVX(m, i, j) * (vx[o] - dt * m->bx[o] * dplus(p, Nx, Nz, i, j, 0, m->c, M, dx));
            vz[o] = DVZ(m, i, j) * (vz[o] - dt * m->bz[o] * dplus(p, Nx, Nz, i, j, 1, m->c, M, dx));
        }
#pragma omp parallel for schedule(static)
    for (int j = 0; j < Nz; ++j)
        for (int i = 0; i < Nx; ++i) {
            size_t o = (size_t)j * Nx + i;
            double dv = dminus(vx, Nx, Nz, i, j, 0, m->c, M, dx) +
                        dminus(vz, Nx, Nz, i, j, 1, m->c, M, dx);
            if (divv) divv[o] = dv;
            p[o] = DP(m, i, j) * (p[o] - dt * m->K[o] * dv);
        }
    for (int c = 0; c < 4; ++c)
        p[sidx[c]] += dt * m->K[sidx[c]] * wn * sw[c] / (dx * dx);
}

static double sample(const double *p, const long *ridx, const double *rw)
{
    double s = 0.0;
    for (int c = 0; c < 4; ++c) s += rw[c] * p[ridx[c]];
    return s;
}

static int geometry(const og_grid *g, int n, const double *xy, long *idx, double *w)
{
    for (int k = 0; k < n; ++k)
        if (oracle_weights(g, xy[2 * k], xy[2 * k + 1], idx + 4 * k, w + 4 * k)) return -1;
    return 0;
}

/* --------------------------------------------------------------- fwi_model */

/* Forward modelling of ns shots (one point source per shot, shared receivers):
 * traces [ns][nr][nt], trace sample n = p^{n+1} at the receiver. */
int oracle_model(const og_grid *g, int pz, const double *xi_a, const double *xi_b, int ns,
                 const double *src_xy, const double *wavelet, int nr, const double *rec_xy,
                 double *traces)
{
    model_t m;
    if (model_init(g, pz, xi_a, xi_b, &m)) return -1;
    long *sidx = malloc(4 * sizeof(long) * (ns > 0 ? ns : 1));
    double *sw = malloc(4 * sizeof(double) * (ns > 0 ? ns : 1));
    long *ridx = malloc(4 * sizeof(long) * (nr > 0 ? nr : 1));
    double *rw = malloc(4 * sizeof(double) * (nr > 0 ? nr : 1));
    int rc = 0;
    if (geometry(g, ns, src_xy, sidx, sw) || geometry(g, nr, rec_xy, ridx, rw)) rc = -1;
    double *p = calloc(m.N, sizeof(double)), *vx = calloc(m.N, sizeof(double)),
           *vz = calloc(m.N, sizeof(double));
    for (int s = 0; s < ns && rc == 0; ++s) {
        memset(p, 0, m.N * sizeof(double));
        memset(vx, 0, m.N * sizeof(double));
        memset(vz, 0, m.N * sizeof(double));
        for (int n = 0; n < g->nt; ++n) {
            step_forward(g, &m, p, vx, vz, sidx + 4 * s, sw + 4 * s, wavelet[n], NULL);
            for (int r = 0; r < nr; ++r)
                traces[((size_t)s * nr + r) * g->nt + n] = sample(p, ridx + 4 * r, rw + 4 * r);
        }
    }
    free(p); free(vx); free(vz); free(sidx); free(sw); free(ridx); free(rw);
    model_free(&m);
    return rc;
}

/* Discrete energy of one shot, E^n = 1/2 sum p^n p^n / K + 1/2 sum (vx^{n-1/2} vx^{n+1/2}/bx +
 * vz^{n-1/2} vz^{n+1/2}/bz), for n = 0 .. nt-1 (sums over cells, unit cell area). */
int oracle_energy(const og_grid *g, int pz, const double *xi_a, const double *xi_b,
                  const double *src_xy, const double *wavelet, double *energy)
{
    model_t m;
    if (model_init(g, pz, xi_a, xi_b, &m)) return -1;
    long sidx[4];
    double sw[4];
    if (geometry(g, 1, src_xy, sidx, sw)) { model_free(&m); return -1; }
    double *p = calloc(m.N, sizeof(double)), *vx = calloc(m.N, sizeof(double)),
           *vz = calloc(m.N, sizeof(double)), *p0 = malloc(m.N * sizeof(double)),
           *vx0 = malloc(m.N * sizeof(double)), *vz0 = malloc(m.N * sizeof(double));
    for (int n = 0; n < g->nt; ++n) {
        memcpy(p0, p, m.N * sizeof(double));
        memcpy(vx0, vx, m.N * sizeof(double));
        memcpy(vz0, vz, m.N * sizeof(double));
        step_forward(g, &m, p, vx, vz, sidx, sw, wavelet[n], NULL);
        double e = 0.0;
        for (size_t o = 0; o < m.N; ++o)
            e += 0.5 * p0[o] * p0[o] / m.K[o] + 0.5 * (vx0[o] * vx[o] / m.bx[o] + vz0[o] * vz[o] / m.bz[o]);
        energy[n] = e;
    }
    free(p); free(vx); free(vz); free(p0); free(vx0); free(vz0);
    model_free(&m);
    return 0;
}

/* ---------------------------------------------------------------- fwi_born */

/* Born modelling: the exact derivative of the forward traces w.r.t. the contrasts along
 * (dxi_a, dxi_b), stepped together with the background wavefield. */
int oracle_born(const og_grid *g, int pz, const double *xi_a, const double *xi_b,
                const double *dxi_a, const double *dxi_b, int ns, const double *src_xy,
                const double *wavelet, int nr, const double *rec_xy, double *dtraces)
{
    model_t m;
    if (model_init(g, pz, xi_a, xi_b, &m)) return -1;
    const int S = m.S, Nx = m.Nx, Nz = m.Nz, M = m.M;
    const double dt = g->dt, dx = g->dx;
    int rc = 0;
    /* perturbations dK, drho on the padded grid (same copy rule as the model), then dbx, dbz */
    double *dK = malloc(m.N * sizeof(double)), *drho = malloc(m.N * sizeof(double)),
           *dbx = malloc(m.N * sizeof(double)), *dbz = malloc(m.N * sizeof(double));
    for (int j = 0; j < Nz && rc == 0; ++j)
        for (int i = 0; i < Nx; ++i) {
            int pi = clampi(i - S, 0, g->nx - 1), pj = clampi(j - S, 0, g->nz - 1);
            size_t q = (size_t)pj * g->nx + pi, o = (size_t)j * Nx + i;
            double jac[4];
            if (jacobian(pz, xi_a[q], xi_b[q], g->vp_o, g->rho_o, jac)) { rc = -1; break; }
            dK[o] = jac[0] * dxi_a[q] + jac[1] * dxi_b[q];
            drho[o] = jac[2] * dxi_a[q] + jac[3] * dxi_b[q];
        }
    for (int j = 0; j < Nz; ++j)
        for (int i = 0; i < Nx; ++i) {
            size_t o = (size_t)j * Nx + i;
            int ir = i + 1 < Nx ? i + 1 : i, jr = j + 1 < Nz ? j + 1 : j;
            size_t ox = (size_t)j * Nx + ir, oz = (size_t)jr * Nx + i;
            /* bx = 2/(rho_o + rho_x): dbx = -bx^2/2 (drho_o + drho_x) */
            dbx[o] = -0.5 * m.bx[o] * m.bx[o] * (drho[o] + drho[ox]);
            dbz[o] = -0.5 * m.bz[o] * m.bz[o] * (drho[o] + drho[oz]);
        }
    long *sidx = malloc(4 * sizeof(long) * (ns > 0 ? ns : 1));
    double *sw = malloc(4 * sizeof(double) * (ns > 0 ? ns : 1));
    long *ridx = malloc(4 * sizeof(long) * (nr > 0 ? nr : 1));
    double *rw = malloc(4 * sizeof(double) * (nr > 0 ? nr : 1));
    if (geometry(g, ns, src_xy, sidx, sw) || geometry(g, nr, rec_xy, ridx, rw)) rc = -1;
    double *p = malloc(m.N * sizeof(double)), *vx = malloc(m.N * sizeof(double)),
           *vz = malloc(m.N * sizeof(double)), *dp = malloc(m.N * sizeof(double)),
           *dvx = malloc(m.N * sizeof(double)), *dvz = malloc(m.N * sizeof(double)),
           *divv = malloc(m.N * sizeof(double));
    for (int s = 0; s < ns && rc == 0; ++s) {
        memset(p, 0, m.N * sizeof(double));  memset(vx, 0, m.N * sizeof(double));
        memset(vz, 0, m.N * sizeof(double)); memset(dp, 0, m.N * sizeof(double));
        memset(dvx, 0, m.N * sizeof(double)); memset(dvz, 0, m.N * sizeof(double));
        const long *si = sidx + 4 * s;
        const double *swt = sw + 4 * s;
        for (int n = 0; n < g->nt; ++n) {
            /* velocities: dv uses dp^n and p^n, both before their updates */
#pragma omp parallel for schedule(static)
            for (int j = 0; j < Nz; ++j)
                for (int i = 0; i < Nx; ++i) {
                    size_t o = (size_t)j * Nx + i;
                    double gpx = dplus(p, Nx, Nz, i, j, 0, m.c, M, dx);
                    double gpz = dplus(p, Nx, Nz, i, j, 1, m.c, M, dx);
                    double gdx = dplus(dp, Nx, Nz, i, j, 0, m.c, M, dx);
                    double gdz = dplus(dp, Nx, Nz, i, j, 1, m.c, M, dx);
                    dvx[o] = DVX(&m, i, j) * (dvx[o] - dt * m.bx[o] * gdx - dt * dbx[o] * gpx);
                    dvz[o] = DVZ(&m, i, j) * (dvz[o] - dt * m.bz[o] * gdz - dt * dbz[o] * gpz);
                    vx[o] = DVX(&m, i, j) * (vx[o] - dt * m.bx[o] * gpx);
                    vz[o] = DVZ(&m, i, j) * (vz[o] - dt * m.bz[o] * gpz);
                }
            /* pressures: dp uses v^{n+1/2} and dv^{n+1/2} */
#pragma omp parallel for schedule(static)
            for (int j = 0; j < Nz; ++j)
                for (int i = 0; i < Nx; ++i) {
                    size_t o = (size_t)j * Nx + i;
                    double d0 = dminus(vx, Nx, Nz, i, j, 0, m.c, M, dx) + dminus(vz, Nx, Nz, i, j, 1, m.c, M, dx);
                    double d1 = dminus(dvx, Nx, Nz, i, j, 0, m.c, M, dx) + dminus(dvz, Nx, Nz, i, j, 1, m.c, M, dx);
                    divv[o] = d0;
                    dp[o] = DP(&m, i, j) * (dp[o] - dt * m.K[o] * d1 - dt * dK[o] * d0);
                    p[o] = DP(&m, i, j) * (p[o] - dt * m.K[o] * d0);
                }
            for (int c = 0; c < 4; ++c) {
                p[si[c]] += dt * m.K[si[c]] * wavelet[n] * swt[c] / (dx * dx);
                dp[si[c]] += dt * dK[si[c]] * wavelet[n] * swt[c] / (dx * dx);
            }
            for (int r = 0; r < nr; ++r)
                dtraces[((size_t)s * nr + r) * g->nt + n] = sample(dp, ridx + 4 * r, rw + 4 * r);
        }
    }
    free(p); free(vx); free(vz); free(dp); free(dvx); free(dvz); free(divv);
    free(dK); free(drho); free(dbx); free(dbz);
    free(sidx); free(sw); free(ridx); free(rw);
    model_free(&m);
    return rc;
}

/* ------------------------------------------------------------- fwi_adjoint */

/* Adjoint modelling and gradient.  For a residual r[ns][nr][nt] (the derivative of the misfit
 * w.r.t. the traces) computes the gradient of sum_{s,r,n} r * trace w.r.t. the contrasts of
 * every parameterization, grads [5][2][nz][nx] (physical grid), and optionally the gradients
 * w.r.t. K and rho on the physical grid (gKrho [2][nz][nx], may be NULL).
 *
 * Per shot the forward run stores p^n and (Dx- vx + Dz- vz)^{n+1/2} for every step; the
 * backward loop then takes the transpose of each forward operation in reverse order:
 *   pbar^{n+1} += R^T r_n                       (trace sampling)
 *   gK_c       += pbar^{n+1}_c dt w_n beta_c/dx^2 (source injection scales with K)
 *   q           = d_p pbar^{n+1}
 *   gK         += q (-dt divv^{n+1/2})
 *   vbar^{n+1/2} += dt D+ (K q)                 (D- transposed is -D+)
 *   u           = d_v vbar^{n+1/2};  gb += u (-dt D+ p^n)
 *   pbar^n      = q + dt D- (b u);   vbar^{n-1/2} = u
 * then g_rho from g_bx, g_bz through bx = 2/(rho_i + rho_{i+1}), the padding cells fold back
 * onto the physical cell they copy, and the chain rule maps (g_K, g_rho) to each pair. */
int oracle_adjoint(const og_grid *g, int pz, const double *xi_a, const double *xi_b, int ns,
                   const double *src_xy, const double *wavelet, int nr, const double *rec_xy,
                   const double *residual, double *grads, double *gKrho)
{
    model_t m;
    if (model_init(g, pz, xi_a, xi_b, &m)) return -1;
    const int S = m.S, Nx = m.Nx, Nz = m.Nz, M = m.M, nt = g->nt;
    const double dt = g->dt, dx = g->dx;
    const size_t N = m.N;
    int rc = 0;
    long *sidx = malloc(4 * sizeof(long) * (ns > 0 ? ns : 1));
    double *sw = malloc(4 * sizeof(double) * (ns > 0 ? ns : 1));
    long *ridx = malloc(4 * sizeof(long) * (nr > 0 ? nr : 1));
    double *rw = malloc(4 * sizeof(double) * (nr > 0 ? nr : 1));
    if (geometry(g, ns, src_xy, sidx, sw) || geometry(g, nr, rec_xy, ridx, rw)) rc = -1;

    double *gK = calloc(N, sizeof(double)), *gbx = calloc(N, sizeof(double)),
           *gbz = calloc(N, sizeof(double));
    double *phist = malloc(N * sizeof(double) * (size_t)(nt > 0 ? nt : 1));
    double *dhist = malloc(N * sizeof(double) * (size_t)(nt > 0 ? nt : 1));
    double *p = malloc(N * sizeof(double)), *vx = malloc(N * sizeof(double)),
           *vz = malloc(N * sizeof(double));
    double *lp = malloc(N * sizeof(double)), *lvx = malloc(N * sizeof(double)),
           *lvz = malloc(N * sizeof(double)), *kq = malloc(N * sizeof(double)),
           *bux = malloc(N * sizeof(double)), *buz = malloc(N * sizeof(double));
    if (!phist || !dhist) rc = -1;

    for (int s = 0; s < ns && rc == 0; ++s) {
        const long *si = sidx + 4 * s;
        const double *swt = sw + 4 * s;
        /* forward, keeping p^n and divv^{n+1/2} */
        memset(p, 0, N * sizeof(double));
        memset(vx, 0, N * sizeof(double));
        memset(vz, 0, N * sizeof(double));
        for (int n = 0; n < nt; ++n) {
            memcpy(phist + (size_t)n * N, p, N * sizeof(double));
            step_forward(g, &m, p, vx, vz, si, swt, wavelet[n], dhist + (size_t)n * N);
        }
        /* backward */
        memset(lp, 0, N * sizeof(double));
        memset(lvx, 0, N * sizeof(double));
        memset(lvz, 0, N * sizeof(double));
        for (int n = nt - 1; n >= 0; --n) {
            for (int r = 0; r < nr; ++r) {
                double rv = residual[((size_t)s * nr + r) * nt + n];
                for (int c = 0; c < 4; ++c) lp[ridx[4 * r + c]] += rw[4 * r + c] * rv;
            }
            for (int c = 0; c < 4; ++c)
                gK[si[c]] += lp[si[c]] * dt * wavelet[n] * swt[c] / (dx * dx);
            const double *divv = dhist + (size_t)n * N, *pn = phist + (size_t)n * N;
#pragma omp parallel for schedule(static)
            for (int j = 0; j < Nz; ++j)
                for (int i = 0; i < Nx; ++i) {
                    size_t o = (size_t)j * Nx + i;
                    double q = DP(&m, i, j) * lp[o];
                    gK[o] += q * (-dt * divv[o]);
                    lp[o] = q;                     /* pbar^n starts with q */
                    kq[o] = m.K[o] * q;
                }
#pragma omp parallel for schedule(static)
            for (int j = 0; j < Nz; ++j)
                for (int i = 0; i < Nx; ++i) {
                    size_t o = (size_t)j * Nx + i;
                    double vbx = lvx[o] + dt * dplus(kq, Nx, Nz, i, j, 0, m.c, M, dx);
                    double vbz = lvz[o] + dt * dplus(kq, Nx, Nz, i, j, 1, m.c, M, dx);
                    double ux = DVX(&m, i, j) * vbx, uz = DVZ(&m, i, j) * vbz;
                    gbx[o] += ux * (-dt * dplus(pn, Nx, Nz, i, j, 0, m.c, M, dx));
                    gbz[o] += uz * (-dt * dplus(pn, Nx, Nz, i, j, 1, m.c, M, dx));
                    lvx[o] = ux;
                    lvz[o] = uz;
                    bux[o] = m.bx[o] * ux;
                    buz[o] = m.bz[o] * uz;
                }
#pragma omp parallel for schedule(static)
            for (int j = 0; j < Nz; ++j)
                for (int i = 0; i < Nx; ++i) {
                    size_t o = (size_t)j * Nx + i;
                    lp[o] += dt * (dminus(bux, Nx, Nz, i, j, 0, m.c, M, dx) +
                                   dminus(buz, Nx, Nz, i, j, 1, m.c, M, dx));
                }
        }
    }

    if (rc == 0) {
        /* g_rho on the padded grid: each buoyancy node depends on its two cells */
        double *grho = calloc(N, sizeof(double));
        for (int j = 0; j < Nz; ++j)
            for (int i = 0; i < Nx; ++i) {
                size_t o = (size_t)j * Nx + i;
                int ir = i + 1 < Nx ? i + 1 : i, jr = j + 1 < Nz ? j + 1 : j;
                double hx = -0.5 * m.bx[o] * m.bx[o] * gbx[o];
                double hz = -0.5 * m.bz[o] * m.bz[o] * gbz[o];
                grho[o] += hx;
                grho[(size_t)j * Nx + ir] += hx;
                grho[o] += hz;
                grho[(size_t)jr * Nx + i] += hz;
            }
        /* fold the padding back onto the physical cells it copies */
        const size_t np = (size_t)g->nx * g->nz;
        double *fK = calloc(np, sizeof(double)), *fr = calloc(np, sizeof(double));
        double *Kp = malloc(np * sizeof(double)), *rp = malloc(np * sizeof(double));
        for (int j = 0; j < Nz; ++j)
            for (int i = 0; i < Nx; ++i) {
                int pi = clampi(i - S, 0, g->nx - 1), pj = clampi(j - S, 0, g->nz - 1);
                size_t q = (size_t)pj * g->nx + pi, o = (size_t)j * Nx + i;
                fK[q] += gK[o];
                fr[q] += grho[o];
            }
        for (int j = 0; j < g->nz; ++j)
            for (int i = 0; i < g->nx; ++i) {
                size_t q = (size_t)j * g->nx + i, o = (size_t)(j + S) * Nx + (i + S);
                Kp[q] = m.K[o];
                rp[q] = m.rho[o];
            }
        if (gKrho) {
            memcpy(gKrho, fK, np * sizeof(double));
            memcpy(gKrho + np, fr, np * sizeof(double));
        }
        if (grads) rc = oracle_chain_rule(g->vp_o, g->rho_o, (int)np, Kp, rp, fK, fr, grads);
        free(grho); free(fK); free(fr); free(Kp); free(rp);
    }
    free(gK); free(gbx); free(gbz); free(phist); free(dhist);
    free(p); free(vx); free(vz); free(lp); free(lvx); free(lvz); free(kq); free(bux); free(buz);
    free(sidx); free(sw); free(ridx); free(rw);
    model_free(&m);
    return rc;
}

/* ------------------------------------------------------------ fwi_gradient */

/* Misfit J = 1/2 sum (d_mod - d_obs)^2 (time-domain reading of the paper's least-squares
 * misfit) and its gradient for all five parameterizations. */
int oracle_gradient(const og_grid *g, int pz, const double *xi_a, const double *xi_b, int ns,
                    const double *src_xy, const double *wavelet, int nr, const double *rec_xy,
                    const double *data, double *misfit, double *grads, double *gKrho)
{
    size_t nd = (size_t)ns * nr * g->nt;
    double *tr = malloc((nd ? nd : 1) * sizeof(double));
    int rc = oracle_model(g, pz, xi_a, xi_b, ns, src_xy, wavelet, nr, rec_xy, tr);
    if (rc == 0) {
        double J = 0.0;
        for (size_t k = 0; k < nd; ++k) {
            tr[k] -= data[k];
            J += 0.5 * tr[k] * tr[k];
        }
        *misfit = J;
        rc = oracle_adjoint(g, pz, xi_a, xi_b, ns, src_xy, wavelet, nr, rec_xy, tr, grads, gKrho);
    }
    free(tr);
    return rc;
}
