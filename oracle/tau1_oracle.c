/*
 * tau1_oracle.c - plain, slow, obviously correct FP64 CPU oracle for the
 * Tau1 lattice Boltzmann update and for standard BGK with stored
 * populations.
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it. The CUDA library never calls it and
 * shares no code, header, table or constant with it.
 *
 * Paper: Bacza, Tomczak, Matyka, "The lattice Boltzmann method for fluid
 * flows at relaxation time equal one: performance study" (arXiv 2312.14742).
 *
 *   Eq. (feq)        f_k^eq = w_k rho (1 + 3 c_k.u + 4.5 (c_k.u)^2 - 1.5 u.u)
 *                    with c_s^2 = 1/3 in lattice units.
 *   Eq. (LBGK)       f_k(x + c_k, t+1) = f_k + (f_k^eq - f_k)/tau.
 *   Eq. (LBMTau1)    at tau = 1: f_k(x + c_k, t+1) = f_k^eq(x, t).
 *   Eqs. (Tau1 density / velocity): the new rho and momentum at x are sums,
 *                    over directions, of the equilibria of the neighbours
 *                    x - c_k evaluated in direction k.
 *   Algorithm "Complete Tau1 ... halfway bounce-back": a link whose source
 *                    x - c_k is a wall takes f^eq_{inv k} of the node's own
 *                    previous (rho*, u*).
 *   Algorithm "Optimized Tau1 ... stores velocity": u is stored, and the
 *                    momentum is multiplied once by r = 1/rho.
 *   Algorithm "Standard LBM" (pull, AB): gather f_k from x - c_k, moments,
 *                    equilibrium, relax, store.
 *
 * Readings fixed here (the paper is silent or ambiguous on these):
 *  - Lattices D2Q9 (one plane, nz = 1), D3Q19 and D3Q27 with the textbook
 *    velocities and weights (Qian et al. 1992).
 *  - A bounced link adds c_k * f^eq_{inv k}(own rho*, own u*): the reflected
 *    population travels along c_k.
 *  - Body force: velocity shift. Every equilibrium is evaluated at
 *    v = u + tau*g (tau = 1 for Tau1); the stored u is the momentum of the
 *    arriving populations over rho, the physical velocity is u + g/2.
 *  - The state is stored as drho = rho - 1 and u. Each equilibrium is
 *    evaluated as its deviation from the rest weight,
 *        f_k^eq - w_k = w_k (drho + rho (3 c_k.v + 4.5 (c_k.v)^2 - 1.5 v.v)),
 *    which is Eq. (feq) exactly, rewritten with sum_k w_k = 1 and
 *    sum_k w_k c_k = 0 so that drho' = sum_k (f_k - w_k) and
 *    j' = sum_k c_k (f_k - w_k) carry no rounding from the constant 1.
 *  - A link that leaves the box across a non-periodic axis counts as a wall.
 *  - Solid nodes hold drho = 0, u = 0 and are never updated.
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off [-fopenmp].
 * -ffp-contract=off keeps every product and sum a separately rounded IEEE
 * operation, so results are the same on every host. OpenMP splits the outer
 * z loop only; each node's arithmetic is unchanged.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- lattices (textbook D3Q19 / D3Q27) --------------------------------- */

typedef struct {
    int q;
    int c[27][3];
    double w[27];
    int inv[27];
} lattice;

/* Velocities: rest, 6 faces, 12 edges, 8 corners, each +/- pair adjacent. */
static const int VEL27[27][3] = {
    { 0, 0, 0},
    { 1, 0, 0}, {-1, 0, 0}, { 0, 1, 0}, { 0,-1, 0}, { 0, 0, 1}, { 0, 0,-1},
    { 1, 1, 0}, {-1,-1, 0}, { 1,-1, 0}, {-1, 1, 0},
    { 1, 0, 1}, {-1, 0,-1}, { 1, 0,-1}, {-1, 0, 1},
    { 0, 1, 1}, { 0,-1,-1}, { 0, 1,-1}, { 0,-1, 1},
    { 1, 1, 1}, {-1,-1,-1}, { 1, 1,-1}, {-1,-1, 1},
    { 1,-1, 1}, {-1, 1,-1}, {-1, 1, 1}, { 1,-1,-1},
};

/* D2Q9 (the plane z = const): rest, 4 axis directions, 4 diagonals. */
static const int VEL9[9][3] = {
    { 0, 0, 0}, { 1, 0, 0}, {-1, 0, 0}, { 0, 1, 0}, { 0,-1, 0},
    { 1, 1, 0}, {-1,-1, 0}, { 1,-1, 0}, {-1, 1, 0},
};

static int lattice_make(int q, lattice* L)
{
    /* weights by squared speed |c|^2 = 0,1,2,3 */
    static const double W9[4] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0, 0.0};
    static const double W19[4] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0, 0.0};
    static const double W27[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
    const double* W;
    const int (*V)[3] = VEL27;
    if (q == 9) { W = W9; V = VEL9; }
    else if (q == 19) W = W19;
    else if (q == 27) W = W27;
    else return -1;
    L->q = q;
    for (int k = 0; k < q; ++k) {
        int s = 0;
        for (int a = 0; a < 3; ++a) { L->c[k][a] = V[k][a]; s += V[k][a] * V[k][a]; }
        L->w[k] = W[s];
    }
    /* opposite direction found by search, not by position */
    for (int k = 0; k < q; ++k) {
        L->inv[k] = -1;
        for (int m = 0; m < q; ++m)
            if (L->c[m][0] == -L->c[k][0] && L->c[m][1] == -L->c[k][1] && L->c[m][2] == -L->c[k][2])
                L->inv[k] = m;
        if (L->inv[k] < 0) return -1;
    }
    return 0;
}

int orc_lattice(int q, int* c, double* w, int* inv)
{
    lattice L;
    if (lattice_make(q, &L)) return -1;
    for (int k = 0; k < q; ++k) {
        for (int a = 0; a < 3; ++a) c[3 * k + a] = L.c[k][a];
        w[k] = L.w[k];
        inv[k] = L.inv[k];
    }
    return 0;
}

/* ---- equilibrium, Eq. (feq), as deviation from w_k ---------------------- */

static double feq_dev(const lattice* L, int k, double drho, double vx, double vy, double vz)
{
    double rho = 1.0 + drho;
    double cu = (double)L->c[k][0] * vx + (double)L->c[k][1] * vy + (double)L->c[k][2] * vz;
    double vv = vx * vx + vy * vy + vz * vz;
    return L->w[k] * (drho + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * vv));
}

double orc_feq_dev(int q, int k, double drho, double vx, double vy, double vz)
{
    lattice L;
    if (lattice_make(q, &L) || k < 0 || k >= q) return NAN;
    return feq_dev(&L, k, drho, vx, vy, vz);
}

/* ---- geometry helpers ---------------------------------------------------- */

typedef struct {
    int nx, ny, nz;
    int periodic[3];
    const uint8_t* solid;
} grid;

static size_t idx3(const grid* G, int x, int y, int z)
{
    return (size_t)x + (size_t)G->nx * ((size_t)y + (size_t)G->ny * (size_t)z);
}

/* Source node x - c_k. Returns 0 and sets *s when it is a fluid node inside
 * the (periodically wrapped) box, 1 when the link is a wall. */
static int link_source(const grid* G, const lattice* L, int k, int x, int y, int z, size_t* s)
{
    int p[3] = {x - L->c[k][0], y - L->c[k][1], z - L->c[k][2]};
    int n[3] = {G->nx, G->ny, G->nz};
    for (int a = 0; a < 3; ++a) {
        if (p[a] < 0 || p[a] >= n[a]) {
            if (!G->periodic[a]) return 1;
            p[a] = (p[a] % n[a] + n[a]) % n[a];
        }
    }
    *s = idx3(G, p[0], p[1], p[2]);
    return G->solid[*s] ? 1 : 0;
}

/* ---- Tau1: one node -------------------------------------------------------
 * Algorithms "Tau1" (pull, AB), "Complete Tau1 with halfway bounce-back" and
 * "Optimized Tau1 that stores velocity": accumulate, over k in order
 * 0..q-1, the equilibrium arriving along c_k, then one reciprocal of rho.
 */
/* The population arriving at (x, y, z) = node i along c_k: the equilibrium
 * of the source x - c_k, or, for a wall link, halfway bounce-back of the
 * node's own previous rho*, u* in direction inv(k). */
static double arriving(const grid* G, const lattice* L, const double g[3],
                       const double* drho, const double* ux, const double* uy, const double* uz,
                       int k, int x, int y, int z, size_t i)
{
    size_t s;
    double f;
    if (link_source(G, L, k, x, y, z, &s)) {
        f = feq_dev(L, L->inv[k], drho[i], ux[i] + g[0], uy[i] + g[1], uz[i] + g[2]);
    } else {
        f = feq_dev(L, k, drho[s], ux[s] + g[0], uy[s] + g[1], uz[s] + g[2]);
    }
    return f;
}

/* Constant-density (pressure) boundaries of Zou and He on the two faces of
 * one non-periodic axis: bc = {axis (or -1: none), rho at coordinate 0,
 * rho at coordinate n-1}. A fluid node on such a face keeps the given
 * density; the populations entering from outside (c_axis pointing into the
 * box) are unknown, the others arrive as in the interior (from fluid
 * sources, or reflected at walls). Zou and He set the unknowns so that the
 * node's moments are (rho_b, u) with u along the axis and
 *     rho_b (1 - s u) = sum_{c_axis = 0} f + 2 sum_{c_axis = -s} f,
 * s = +1 on the low face (inflow along +axis) and -1 on the high face, and
 * the transverse velocity is zero. At tau = 1 the node's new state is those
 * moments, so Tau1 needs only the known sums. With f = w + h (h the
 * deviation) and sum_{c_axis=0} w + 2 sum_{c_axis=-s} w = 1:
 *     u = s (rho_b - 1 - H0 - 2 Hout) / rho_b.
 */
static int zou_he_node(const grid* G, const lattice* L, const double g[3], const double* bc,
                       const double* drho, const double* ux, const double* uy, const double* uz,
                       int x, int y, int z, double out[4])
{
    int a = (int)bc[0];
    if (a < 0 || a > 2) return 0;
    int pos[3] = {x, y, z};
    int n[3] = {G->nx, G->ny, G->nz};
    double sgn;
    double rho_b;
    if (pos[a] == 0) { sgn = 1.0; rho_b = bc[1]; }
    else if (pos[a] == n[a] - 1) { sgn = -1.0; rho_b = bc[2]; }
    else return 0;
    size_t i = idx3(G, x, y, z);
    double h0 = 0.0, hout = 0.0;
    for (int k = 0; k < L->q; ++k) {
        int ck = L->c[k][a];
        if ((double)ck == sgn) continue; /* unknown: enters from outside */
        double f = arriving(G, L, g, drho, ux, uy, uz, k, x, y, z, i);
        if (ck == 0) h0 += f;
        else hout += f;
    }
    double u = sgn * ((rho_b - 1.0) - h0 - 2.0 * hout) / rho_b;
    out[0] = rho_b - 1.0;
    out[1] = out[2] = out[3] = 0.0;
    out[1 + a] = u;
    return 1;
}

static void tau1_node(const grid* G, const lattice* L, const double g[3], const double* bc,
                      const double* drho, const double* ux, const double* uy, const double* uz,
                      int x, int y, int z, double out[4])
{
    size_t i = idx3(G, x, y, z);
    if (G->solid[i]) { out[0] = out[1] = out[2] = out[3] = 0.0; return; }
    if (bc && zou_he_node(G, L, g, bc, drho, ux, uy, uz, x, y, z, out)) return;
    double d_acc = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int k = 0; k < L->q; ++k) {
        double f = arriving(G, L, g, drho, ux, uy, uz, k, x, y, z, i);
        d_acc += f;
        jx += (double)L->c[k][0] * f;
        jy += (double)L->c[k][1] * f;
        jz += (double)L->c[k][2] * f;
    }
    double r = 1.0 / (1.0 + d_acc);
    out[0] = d_acc;
    out[1] = jx * r;
    out[2] = jy * r;
    out[3] = jz * r;
}

static int check_args(int q, int nx, int ny, int nz, lattice* L)
{
    if (nx <= 0 || ny <= 0 || nz <= 0) return -1;
    if (q == 9 && nz != 1) return -1; /* D2Q9: one plane */
    return lattice_make(q, L);
}

/* A pressure boundary needs a non-periodic axis of the box (NULL: none). */
static int check_bc(const double* bc, const int* periodic)
{
    if (!bc || bc[0] < 0.0) return 0;
    int a = (int)bc[0];
    if (a > 2 || periodic[a] || !(bc[1] > 0.0) || !(bc[2] > 0.0)) return -1;
    return 0;
}

/* One Tau1 step over the whole box: (drho,ux,uy,uz) -> (*_o), with optional
 * pressure faces bc (see zou_he_node; NULL or bc[0] < 0: none). */
int orc_tau1_step_bc(int q, int nx, int ny, int nz, const int* periodic, const double* g, const double* bc,
                     const uint8_t* solid,
                     const double* drho, const double* ux, const double* uy, const double* uz,
                     double* drho_o, double* ux_o, double* uy_o, double* uz_o)
{
    lattice L;
    if (check_args(q, nx, ny, nz, &L) || check_bc(bc, periodic)) return -1;
    if (bc && bc[0] < 0.0) bc = NULL;
    grid G = {nx, ny, nz, {periodic[0], periodic[1], periodic[2]}, solid};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double o[4];
                tau1_node(&G, &L, g, bc, drho, ux, uy, uz, x, y, z, o);
                size_t i = idx3(&G, x, y, z);
                drho_o[i] = o[0]; ux_o[i] = o[1]; uy_o[i] = o[2]; uz_o[i] = o[3];
            }
    return 0;
}

int orc_tau1_step(int q, int nx, int ny, int nz, const int* periodic, const double* g,
                  const uint8_t* solid,
                  const double* drho, const double* ux, const double* uy, const double* uz,
                  double* drho_o, double* ux_o, double* uy_o, double* uz_o)
{
    return orc_tau1_step_bc(q, nx, ny, nz, periodic, g, NULL, solid, drho, ux, uy, uz, drho_o, ux_o, uy_o, uz_o);
}

/* nsteps Tau1 steps in place on (drho,ux,uy,uz), ping-pong with scratch,
 * with optional pressure faces bc. */
int orc_tau1_run_bc(int q, int nx, int ny, int nz, const int* periodic, const double* g, const double* bc,
                    const uint8_t* solid, double* drho, double* ux, double* uy, double* uz,
                    int64_t nsteps)
{
    size_t n = (size_t)nx * (size_t)ny * (size_t)nz;
    double* tmp = (double*)malloc(4 * n * sizeof(double));
    if (!tmp) return -2;
    double* a[4] = {drho, ux, uy, uz};
    double* b[4] = {tmp, tmp + n, tmp + 2 * n, tmp + 3 * n};
    int rc = 0;
    for (int64_t t = 0; t < nsteps && rc == 0; ++t) {
        rc = orc_tau1_step_bc(q, nx, ny, nz, periodic, g, bc, solid, a[0], a[1], a[2], a[3],
                              b[0], b[1], b[2], b[3]);
        for (int f = 0; f < 4; ++f) { double* s = a[f]; a[f] = b[f]; b[f] = s; }
    }
    if (nsteps % 2)  /* result sits in tmp: copy back */
        for (int f = 0; f < 4; ++f) memcpy(b[f], a[f], n * sizeof(double));
    free(tmp);
    return rc;
}

int orc_tau1_run(int q, int nx, int ny, int nz, const int* periodic, const double* g,
                 const uint8_t* solid, double* drho, double* ux, double* uy, double* uz,
                 int64_t nsteps)
{
    return orc_tau1_run_bc(q, nx, ny, nz, periodic, g, NULL, solid, drho, ux, uy, uz, nsteps);
}

/* One Tau1 step evaluated only at the listed flat node indices.
 * out is [count][4] = (drho, ux, uy, uz) of each listed node. */
int orc_tau1_nodes(int q, int nx, int ny, int nz, const int* periodic, const double* g,
                   const uint8_t* solid,
                   const double* drho, const double* ux, const double* uy, const double* uz,
                   const int64_t* nodes, int64_t count, double* out)
{
    lattice L;
    if (check_args(q, nx, ny, nz, &L)) return -1;
    grid G = {nx, ny, nz, {periodic[0], periodic[1], periodic[2]}, solid};
    int64_t n = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < count; ++m) {
        int64_t i = nodes[m];
        if (i < 0 || i >= n) { out[4 * m] = out[4 * m + 1] = out[4 * m + 2] = out[4 * m + 3] = NAN; continue; }
        int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        tau1_node(&G, &L, g, NULL, drho, ux, uy, uz, x, y, z, out + 4 * m);
    }
    return 0;
}

/* ---- standard BGK with stored populations (pull, AB) ---------------------
 * Populations are stored as deviations h_k = f_k - w_k, layout [k][node].
 * The arrays hold post-collision populations of the previous step.
 */

/* Post-collision populations of the initial state: h_k = f_k^eq - w_k at
 * v = u + tau*g, so that the first BGK step sees what Tau1 sees. */
int orc_bgk_init(int q, int nx, int ny, int nz, const double* g, double tau,
                 const uint8_t* solid,
                 const double* drho, const double* ux, const double* uy, const double* uz,
                 double* h)
{
    lattice L;
    if (check_args(q, nx, ny, nz, &L)) return -1;
    size_t n = (size_t)nx * (size_t)ny * (size_t)nz;
    for (size_t i = 0; i < n; ++i)
        for (int k = 0; k < q; ++k)
            h[(size_t)k * n + i] = solid[i] ? 0.0
                : feq_dev(&L, k, drho[i], ux[i] + tau * g[0], uy[i] + tau * g[1], uz[i] + tau * g[2]);
    return 0;
}

/* One BGK step, Algorithm "Standard LBM" with Eq. (LBGK):
 * gather h'_k = h_k(x - c_k) (wall: h_{inv k}(x), halfway bounce-back),
 * moments drho = sum h', j = sum c h', u = j / rho,
 * relax h'' = h' + (h^eq(drho, u + tau*g) - h') / tau, store h''.
 * The moments of the gathered populations are written to (*_o). */
int orc_bgk_step(int q, int nx, int ny, int nz, const int* periodic, const double* g, double tau,
                 const uint8_t* solid, const double* h_in, double* h_out,
                 double* drho_o, double* ux_o, double* uy_o, double* uz_o)
{
    lattice L;
    if (check_args(q, nx, ny, nz, &L) || !(tau > 0.5)) return -1;
    grid G = {nx, ny, nz, {periodic[0], periodic[1], periodic[2]}, solid};
    size_t n = (size_t)nx * (size_t)ny * (size_t)nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = idx3(&G, x, y, z);
                if (solid[i]) {
                    for (int k = 0; k < q; ++k) h_out[(size_t)k * n + i] = 0.0;
                    drho_o[i] = ux_o[i] = uy_o[i] = uz_o[i] = 0.0;
                    continue;
                }
                double hp[27];
                for (int k = 0; k < q; ++k) {
                    size_t s;
                    if (link_source(&G, &L, k, x, y, z, &s))
                        hp[k] = h_in[(size_t)L.inv[k] * n + i];
                    else
                        hp[k] = h_in[(size_t)k * n + s];
                }
                double d = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
                for (int k = 0; k < q; ++k) {
                    d += hp[k];
                    jx += (double)L.c[k][0] * hp[k];
                    jy += (double)L.c[k][1] * hp[k];
                    jz += (double)L.c[k][2] * hp[k];
                }
                double rho = 1.0 + d;
                double vx = jx / rho, vy = jy / rho, vz = jz / rho;
                for (int k = 0; k < q; ++k) {
                    double heq = feq_dev(&L, k, d, vx + tau * g[0], vy + tau * g[1], vz + tau * g[2]);
                    h_out[(size_t)k * n + i] = hp[k] + (heq - hp[k]) / tau;
                }
                drho_o[i] = d; ux_o[i] = vx; uy_o[i] = vy; uz_o[i] = vz;
            }
    return 0;
}

/* ---- global reductions ----------------------------------------------------
 * out[0] fluid node count, out[1] mass sum_fluid (1 + drho),
 * out[2] superficial mean of the physical u_x: sum_fluid (u_x + g_x/2) / N,
 * out[3..5] fluid mean of the physical velocity u + g/2,
 * out[6] max over fluid nodes of |u + g/2|,
 * out[7] permeability nu * out[2] / g_x with nu = 1/6 (Darcy; NaN if g_x = 0),
 * out[8] count of fluid nodes holding a non-finite value.
 */
int orc_reduce(int nx, int ny, int nz, const double* g, const uint8_t* solid,
               const double* drho, const double* ux, const double* uy, const double* uz,
               double* out)
{
    size_t n = (size_t)nx * (size_t)ny * (size_t)nz;
    double nf = 0, mass = 0, sx = 0, sy = 0, sz = 0, umax = 0, bad = 0;
    for (size_t i = 0; i < n; ++i) {
        if (solid[i]) continue;
        nf += 1.0;
        double px = ux[i] + 0.5 * g[0], py = uy[i] + 0.5 * g[1], pz = uz[i] + 0.5 * g[2];
        if (!isfinite(drho[i]) || !isfinite(px) || !isfinite(py) || !isfinite(pz)) bad += 1.0;
        mass += 1.0 + drho[i];
        sx += px; sy += py; sz += pz;
        double m = sqrt(px * px + py * py + pz * pz);
        if (m > umax) umax = m;
    }
    out[0] = nf;
    out[1] = mass;
    out[2] = sx / (double)n;
    out[3] = nf > 0 ? sx / nf : 0.0;
    out[4] = nf > 0 ? sy / nf : 0.0;
    out[5] = nf > 0 ? sz / nf : 0.0;
    out[6] = umax;
    out[7] = g[0] != 0.0 ? (1.0 / 6.0) * out[2] / g[0] : NAN;
    out[8] = bad;
    return 0;
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
