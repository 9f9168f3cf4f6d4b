/*
 * nh_oracle.c -- plain FP64 CPU oracle for the hybrid lattice-Boltzmann (LB)
 * + finite-difference (FD) nematohydrodynamics time step of Amaral, Sedahmed,
 * Telo da Gama and Coelho, "Efficient single-precision simulations of
 * nematohydrodynamics" (arXiv:2503.06610).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  This is the slow, obviously correct
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or constant with the CUDA library, and it never calls it.
 *
 * Every quantity is double precision.  Every routine visits one site at a time
 * and evaluates the formula the paper writes down, in the paper's notation:
 *
 *   - LB step (Sec. II.C): pull-streaming with half-way bounce-back, moments
 *     (Eqs. shifted-rho / shifeted-u, or the unshifted rho / u equations),
 *     equilibrium (Eq. feq-eq or Eq. shifted-feq), Guo source S_i^F, and the
 *     SRT relaxation of Eq. shifted-lbe (or the unshifted LBE).
 *   - FD director step (Sec. II.B): time derivative of Eq. director-time-eq
 *     with central differences (the first-derivative stencil of Sec. II.B) and
 *     the predictor-corrector scheme listed there, then |n| = 1.
 *   - LC stress and force (Eq. force-lc-eq): sigma at every fluid node, its
 *     central divergence, with zero stress at solid ghost nodes.
 *
 * Where the paper is silent the readings are:
 *   - molecular field in one-constant form with chirality,
 *       h = K lap(n) - 2 K q0 curl(n) + W0 n_z z_hat,
 *     lap = compact 3-point Laplacian per axis, curl = central differences,
 *     written as the exact minus derivative of the lattice energy that the
 *     Python side of the oracle evaluates (a sum over nearest-neighbour
 *     links); a plate without anchoring is a free surface whose links carry
 *     no energy, so at the two plate layers the chiral term lacks its link
 *     to the ghost layer;
 *   - the kinematic transport inside the stress is
 *       N = [h_perp - gamma2 (I - n n) D n] / gamma1,   h_perp = h - (h.n) n,
 *     i.e. the director equation solved for N and projected normal to n;
 *   - ghost layers at z = -1 and z = nz when walls are present: u = 0,
 *     n = z_hat (infinite homeotropic anchoring) or n = adjacent fluid layer
 *     (no anchoring); stress = 0 at the ghosts;
 *   - the FD update renormalises n after the corrector only (renorm_predictor
 *     also renormalises the predictor);
 *   - second derivatives: the compact Laplacian (lap_wide: the central
 *     difference of the central difference, n at distance 2 read with the
 *     same ghost rule as at distance 1);
 *   - N in the stress from the director equation (n_from_rate: dn/dt +
 *     u.grad n - W n as Sec. II.A defines N, with dn/dt the averaged time
 *     derivative of the corrector, Sec. II.B, projected normal to n);
 *   - ghost stress zero (ghost_sigma = 1: the stress of the adjacent layer);
 *   - obstacles (solid nodes, Sec. II.B): a link from a fluid site to a solid
 *     one bounces back half-way like the plates; solid nodes keep their
 *     director (infinite anchoring: the caller stores the surface normal
 *     there), their velocity is zero and their stress is zero; their
 *     populations are carried over unchanged;
 *   - three-constant energy (Eq. free-energy-eq with K11, K22, K33): the
 *     one-constant lattice energy with K plus, at every fluid site,
 *       Delta f = (K11-K)/2 (div n)^2 + (K22-K)/2 (n.curl n + q0)^2
 *               + (K33-K)/2 |n x curl n|^2
 *     with central differences; its molecular field is the exact
 *     -d(sum Delta f)/dn, ghost layers included.
 *
 * Layouts: a scalar field is [N] with site index x + nx*(y + ny*z); a vector
 * field is [3][N]; a tensor field is [9][N] with component a*3+b; populations
 * are [19][N] in the velocity order of E[] below.
 */
#include <math.h>
#include <stdlib.h>
#include <stddef.h>
#include <string.h>

typedef struct {
    int nx, ny, nz;
    int walls_z;      /* 1: no-slip plates half-way below z=0 and above z=nz-1; 0: periodic in z */
    int anchoring;    /* 1: infinite homeotropic (ghost n = z_hat); 0: none (ghost n = adjacent layer) */
    int shifted;      /* 1: populations are f_i - w_i (Eq. shifted-feq); 0: plain f_i */
    double tau;       /* SRT relaxation time */
    double g[3];      /* body acceleration (the rho*g term of Eq. NS-eq) */
    double K, q0, gamma1, gamma2;
    double alpha1, alpha2, alpha3, alpha4p, alpha5, alpha6;  /* alpha4p = alpha_4' of Eq. force-lc-eq */
    double W0;        /* bulk effective anchoring strength */
    double dt_fd;     /* FD time step, in LB time steps */
    double K11, K22, K33; /* three-constant Frank energy (used when frank3 = 1) */
    int frank3;       /* 1: add the three-constant correction Delta f (see frank3_point) */
    const unsigned char* solid; /* [N] 1 = solid node (obstacle), or NULL: no obstacles */
    /* readings where the paper is silent (0 = default) */
    int renorm_predictor; /* 1: the predictor n^P is also renormalised */
    int lap_wide;     /* 1: second derivatives in h as central differences of central differences */
    int n_from_rate;  /* 1: N in the stress from the corrector's averaged rate (see or_stress) */
    int ghost_sigma;  /* 0: zero stress at the plates' ghost layers; 1: the adjacent layer's stress */
} or_params;

/* D3Q19 velocity set (Sec. II.C): rest, 6 axis links, 12 face diagonals. */
static const int E[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static const double CS2 = 1.0 / 3.0; /* c_s^2, c_s = 1/sqrt(3) */

/* Weight by |e_i|^2 (Sec. II.C): 1/3, 1/18, 1/36. */
static double weight(int i)
{
    int e2 = E[i][0] * E[i][0] + E[i][1] * E[i][1] + E[i][2] * E[i][2];
    if (e2 == 0) return 1.0 / 3.0;
    if (e2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* Index of the velocity opposite to e_i, found by search. */
static int opposite(int i)
{
    for (int j = 0; j < 19; ++j)
        if (E[j][0] == -E[i][0] && E[j][1] == -E[i][1] && E[j][2] == -E[i][2]) return j;
    return -1;
}

static int wrap(int a, int n) { return ((a % n) + n) % n; }

static size_t site(const or_params* p, int x, int y, int z)
{
    return (size_t)x + (size_t)p->nx * ((size_t)y + (size_t)p->ny * (size_t)z);
}

static int is_solid(const or_params* p, size_t s) { return p->solid != NULL && p->solid[s] != 0; }

static double levi(int a, int b, int c)
{
    if (a == b || b == c || a == c) return 0.0;
    if ((a == 0 && b == 1 && c == 2) || (a == 1 && b == 2 && c == 0) || (a == 2 && b == 0 && c == 1)) return 1.0;
    return -1.0;
}

/* ---------------------------------------------------------------- lattice */

void or_lattice(int* e_out /* [19*3] */, double* w_out /* [19] */, int* opp_out /* [19] */)
{
    for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a) e_out[3 * i + a] = E[i][a];
        w_out[i] = weight(i);
        opp_out[i] = opposite(i);
    }
}

/* Equilibrium, Eq. feq-eq (shifted = 0) or Eq. shifted-feq (shifted = 1). */
void or_feq(double rho, const double* u, int shifted, double* feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < 19; ++i) {
        double eu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
        double w = weight(i);
        double poly = eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2);
        if (shifted)
            feq[i] = w * rho * poly + (rho - 1.0) * w;
        else
            feq[i] = w * rho * (1.0 + poly);
    }
}

/* Guo source term S_i^F (Sec. II.C). */
void or_guo_source(const double* u, const double* F, double* S)
{
    for (int i = 0; i < 19; ++i) {
        double eF = E[i][0] * F[0] + E[i][1] * F[1] + E[i][2] * F[2];
        double second = 0.0; /* (e_i e_i - c_s^2 I) : (u F + F u) */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double Q = E[i][a] * E[i][b] - (a == b ? CS2 : 0.0);
                second += Q * (u[a] * F[b] + F[a] * u[b]);
            }
        S[i] = weight(i) * (eF / CS2 + second / (2.0 * CS2 * CS2));
    }
}

/* ---------------------------------------------------------------- LB step */

/* One LB time step.  f holds the post-collision populations of the previous
 * step; fnew receives the new post-collision populations.  Streaming is done
 * by pulling f_i from x - e_i; a link that crosses a plate is replaced by the
 * half-way bounce-back f_i(x) <- f_opp(i)(x).  The collision's Guo source uses
 * the force F = F_lc + rho g of the current FD interval.  The velocity
 * u = (sum e_i f_i + H/2)/rho of Eq. shifeted-u takes H = Fu_lc + rho g when
 * Fu_lc is given (the force in effect when the paper's loop computed the
 * macroscopic fields, Sec. II.D), else H = F.  rho and u (the macroscopic
 * fields used by the collision, Eqs. shifted-rho / shifeted-u) are returned. */
void or_lb_step(const or_params* p, const double* f, double* fnew, const double* Flc, const double* Fu_lc,
                double* rho_out, double* u_out)
{
    const size_t N = (size_t)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t s = site(p, x, y, z);
                double fin[19];
                if (is_solid(p, s)) {
                    /* solid node: populations carried over, u = 0, rho = 1 */
                    for (int i = 0; i < 19; ++i) fnew[(size_t)i * N + s] = f[(size_t)i * N + s];
                    rho_out[s] = 1.0;
                    for (int a = 0; a < 3; ++a) u_out[(size_t)a * N + s] = 0.0;
                    continue;
                }
                /* streaming (pull) with half-way bounce-back at plates and obstacles */
                for (int i = 0; i < 19; ++i) {
                    int zs = z - E[i][2];
                    if (p->walls_z && (zs < 0 || zs >= p->nz)) {
                        fin[i] = f[(size_t)opposite(i) * N + s];
                    } else {
                        int xs = wrap(x - E[i][0], p->nx);
                        int ys = wrap(y - E[i][1], p->ny);
                        size_t src = site(p, xs, ys, wrap(zs, p->nz));
                        fin[i] = is_solid(p, src) ? f[(size_t)opposite(i) * N + s] : f[(size_t)i * N + src];
                    }
                }
                /* macroscopic quantities */
                double sum = 0.0, mom[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < 19; ++i) {
                    sum += fin[i];
                    for (int a = 0; a < 3; ++a) mom[a] += E[i][a] * fin[i];
                }
                double rho = p->shifted ? 1.0 + sum : sum;
                double F[3], H[3], u[3];
                for (int a = 0; a < 3; ++a) F[a] = Flc[(size_t)a * N + s] + rho * p->g[a];
                for (int a = 0; a < 3; ++a) H[a] = (Fu_lc ? Fu_lc[(size_t)a * N + s] + rho * p->g[a] : F[a]);
                for (int a = 0; a < 3; ++a) u[a] = mom[a] / rho + H[a] / (2.0 * rho);
                /* collision */
                double feq[19], S[19];
                or_feq(rho, u, p->shifted, feq);
                or_guo_source(u, F, S);
                for (int i = 0; i < 19; ++i)
                    fnew[(size_t)i * N + s] =
                        fin[i] - (fin[i] - feq[i]) / p->tau + (1.0 - 1.0 / (2.0 * p->tau)) * S[i];
                rho_out[s] = rho;
                for (int a = 0; a < 3; ++a) u_out[(size_t)a * N + s] = u[a];
            }
}

/* Populations at rest or at a given (rho, u): f = f^eq(rho, u). */
void or_init_populations(const or_params* p, const double* rho, const double* u, double* f)
{
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    for (size_t s = 0; s < N; ++s) {
        double uu[3] = {u[s], u[N + s], u[2 * N + s]};
        double feq[19];
        or_feq(rho[s], uu, p->shifted, feq);
        for (int i = 0; i < 19; ++i) f[(size_t)i * N + s] = feq[i];
    }
}

/* ---------------------------------------------------------------- FD */

/* Director at a lattice point, including ghost layers beyond the plates. */
static void n_at(const or_params* p, const double* n, int x, int y, int z, double* out)
{
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    x = wrap(x, p->nx);
    y = wrap(y, p->ny);
    if (p->walls_z && (z < 0 || z >= p->nz)) {
        if (p->anchoring) {
            out[0] = 0.0;
            out[1] = 0.0;
            out[2] = 1.0;
            return;
        }
        z = z < 0 ? 0 : p->nz - 1;
    }
    z = wrap(z, p->nz);
    size_t s = site(p, x, y, z);
    for (int a = 0; a < 3; ++a) out[a] = n[(size_t)a * N + s];
}

/* Velocity at a lattice point; zero at the solid ghost layers (and
 * everywhere when u is NULL, i.e. a fluid at rest). */
static void u_at(const or_params* p, const double* u, int x, int y, int z, double* out)
{
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    if (u == NULL || (p->walls_z && (z < 0 || z >= p->nz))) {
        out[0] = out[1] = out[2] = 0.0;
        return;
    }
    size_t s = site(p, wrap(x, p->nx), wrap(y, p->ny), wrap(z, p->nz));
    if (is_solid(p, s)) {
        out[0] = out[1] = out[2] = 0.0;
        return;
    }
    for (int a = 0; a < 3; ++a) out[a] = u[(size_t)a * N + s];
}

/* Local differential quantities at one fluid site:
 *   dn[b][c] = d_b n_c  (central differences),
 *   lap[c]   = compact Laplacian of n_c,
 *   du[a][b] = d_a u_b  (central differences). */
static void local_derivs(const or_params* p, const double* n, const double* u, int x, int y, int z, double dn[3][3],
                         double lap[3], double du[3][3])
{
    double c[3];
    n_at(p, n, x, y, z, c);
    for (int a = 0; a < 3; ++a) lap[a] = 0.0;
    for (int b = 0; b < 3; ++b) {
        int d[3] = {0, 0, 0};
        d[b] = 1;
        double np[3], nm[3], up[3], um[3];
        n_at(p, n, x + d[0], y + d[1], z + d[2], np);
        n_at(p, n, x - d[0], y - d[1], z - d[2], nm);
        u_at(p, u, x + d[0], y + d[1], z + d[2], up);
        u_at(p, u, x - d[0], y - d[1], z - d[2], um);
        for (int k = 0; k < 3; ++k) {
            dn[b][k] = 0.5 * (np[k] - nm[k]);
            du[b][k] = 0.5 * (up[k] - um[k]);
            if (!p->lap_wide) lap[k] += np[k] + nm[k] - 2.0 * c[k];
        }
        if (p->lap_wide) {
            /* d_b (d_b n) with both derivatives central: [n(x+2e) - 2 n(x) + n(x-2e)]/4 */
            double n2p[3], n2m[3];
            n_at(p, n, x + 2 * d[0], y + 2 * d[1], z + 2 * d[2], n2p);
            n_at(p, n, x - 2 * d[0], y - 2 * d[1], z - 2 * d[2], n2m);
            for (int k = 0; k < 3; ++k) lap[k] += 0.25 * (n2p[k] + n2m[k] - 2.0 * c[k]);
        }
    }
}

/* Does the lattice link between layer z and layer zn (= z +- 1) carry energy?
 * Inside the channel, and towards a plate with infinite homeotropic anchoring
 * (a fixed ghost director), yes.  Towards a plate without anchoring, no: the
 * plate is a free surface, and with the ghost director copied from the
 * adjacent layer the link's elastic and chiral energies are both zero. */
static int link_exists(const or_params* p, int zn)
{
    if (!p->walls_z) return 1;
    if (zn >= 0 && zn < p->nz) return 1;
    return p->anchoring != 0;
}

/* Chiral part of the molecular field at (x, y, z): minus the derivative of the
 * chiral link energy K q0 sum_links eps_abc n_a(x) n_c(x + e_b) with respect
 * to n(x, y, z).  A site is the first end of the link (y, y + e_b) and the
 * second end of the link (y - e_b, y), so
 *   hc_m = -K q0 sum_b [ eps_mbc n_c(y + e_b) + eps_abm n_a(y - e_b) ]
 * over the links that exist.  In the bulk this is -2 K q0 (curl n)_m with
 * the central curl. */
static void chiral_field(const or_params* p, const double* n, int x, int y, int z, double hc[3])
{
    for (int m = 0; m < 3; ++m) hc[m] = 0.0;
    for (int b = 0; b < 3; ++b) {
        int d[3] = {0, 0, 0};
        d[b] = 1;
        double np[3], nm[3];
        if (link_exists(p, z + d[2])) {
            n_at(p, n, x + d[0], y + d[1], z + d[2], np);
            for (int m = 0; m < 3; ++m)
                for (int c = 0; c < 3; ++c) hc[m] -= p->K * p->q0 * levi(m, b, c) * np[c];
        }
        if (link_exists(p, z - d[2])) {
            n_at(p, n, x - d[0], y - d[1], z - d[2], nm);
            for (int m = 0; m < 3; ++m)
                for (int a = 0; a < 3; ++a) hc[m] -= p->K * p->q0 * levi(a, b, m) * nm[a];
        }
    }
}

/* Molecular field h = -dE_d/dn of the one-constant lattice energy (Sec. II.A):
 * h = K lap n + hc + W0 n_z z_hat, with the compact Laplacian (the elastic
 * link energy; a copied ghost contributes nothing) and the chiral part hc of
 * chiral_field (-2 K q0 curl n in the bulk). */
static void molecular_field(const or_params* p, const double* n, int x, int y, int z, const double nc[3],
                            const double lap[3], double h[3])
{
    double hc[3];
    chiral_field(p, n, x, y, z, hc);
    for (int a = 0; a < 3; ++a) h[a] = p->K * lap[a] + hc[a];
    h[2] += p->W0 * nc[2];
}

/* Three-constant correction at one site, from the director nc and its
 * central gradient G[b][c] = d_b n_c (Eq. free-energy-eq minus its
 * one-constant form with K):
 *   div = G_aa,  w_a = eps_abc G_bc (curl),  t = n.w + q0,
 *   Delta f = a1/2 div^2 + a2/2 t^2 + a3/2 (|n|^2 |w|^2 - (n.w)^2),
 *   a1 = K11 - K, a2 = K22 - K, a3 = K33 - K
 * (|n x w|^2 written by Lagrange's identity, valid for any n).  Returns
 * Delta f, dfdn[c] = d Delta f / d n_c and P[b][c] = d Delta f / d G_bc. */
static double frank3_point(const or_params* p, const double nc[3], const double G[3][3], double dfdn[3],
                           double P[3][3])
{
    const double a1 = p->K11 - p->K, a2 = p->K22 - p->K, a3 = p->K33 - p->K;
    double div = G[0][0] + G[1][1] + G[2][2];
    double w[3];
    for (int a = 0; a < 3; ++a) {
        w[a] = 0.0;
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) w[a] += levi(a, b, c) * G[b][c];
    }
    double nw = nc[0] * w[0] + nc[1] * w[1] + nc[2] * w[2];
    double nn = nc[0] * nc[0] + nc[1] * nc[1] + nc[2] * nc[2];
    double ww = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double t = nw + p->q0;
    double V[3];
    for (int c = 0; c < 3; ++c) {
        dfdn[c] = a2 * t * w[c] + a3 * (nc[c] * ww - nw * w[c]);
        V[c] = a2 * t * nc[c] + a3 * (nn * w[c] - nw * nc[c]); /* d Delta f / d w_c */
    }
    for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c) {
            double v = (b == c) ? a1 * div : 0.0;
            for (int a = 0; a < 3; ++a) v += levi(a, b, c) * V[a];
            P[b][c] = v;
        }
    return 0.5 * a1 * div * div + 0.5 * a2 * t * t + 0.5 * a3 * (nn * ww - nw * nw);
}

/* Site that supplies the director at (x, y, z), which may lie in a ghost
 * layer: -1 for a fixed ghost value (homeotropic plates). */
static long n_source(const or_params* p, int x, int y, int z)
{
    x = wrap(x, p->nx);
    y = wrap(y, p->ny);
    if (p->walls_z && (z < 0 || z >= p->nz)) {
        if (p->anchoring) return -1;
        z = z < 0 ? 0 : p->nz - 1;
    }
    return (long)site(p, x, y, wrap(z, p->nz));
}

/* Central gradient G[b][c] = d_b n_c at a fluid site (ghost reading). */
static void central_gradient(const or_params* p, const double* n, int x, int y, int z, double G[3][3])
{
    for (int b = 0; b < 3; ++b) {
        int d[3] = {0, 0, 0};
        d[b] = 1;
        double np[3], nm[3];
        n_at(p, n, x + d[0], y + d[1], z + d[2], np);
        n_at(p, n, x - d[0], y - d[1], z - d[2], nm);
        for (int c = 0; c < 3; ++c) G[b][c] = 0.5 * (np[c] - nm[c]);
    }
}

/* Molecular field of the three-constant correction, hd = -d(sum_x Delta f)/dn,
 * by scattering every site's derivatives onto the sites its gradient reads:
 * G_bc(x) = [n_c(source(x + e_b)) - n_c(source(x - e_b))]/2.  Returns the sum
 * of Delta f.  hd is [3][N]. */
static double frank3_field(const or_params* p, const double* n, double* hd)
{
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    double E = 0.0;
    memset(hd, 0, 3 * N * sizeof(double));
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t s = site(p, x, y, z);
                if (is_solid(p, s)) continue; /* no energy at solid nodes */
                double nc[3], G[3][3], dfdn[3], P[3][3];
                n_at(p, n, x, y, z, nc);
                central_gradient(p, n, x, y, z, G);
                E += frank3_point(p, nc, G, dfdn, P);
                for (int c = 0; c < 3; ++c) hd[(size_t)c * N + s] -= dfdn[c];
                for (int b = 0; b < 3; ++b) {
                    int d[3] = {0, 0, 0};
                    d[b] = 1;
                    long sp = n_source(p, x + d[0], y + d[1], z + d[2]);
                    long sm = n_source(p, x - d[0], y - d[1], z - d[2]);
                    for (int c = 0; c < 3; ++c) {
                        if (sp >= 0) hd[(size_t)c * N + (size_t)sp] -= 0.5 * P[b][c];
                        if (sm >= 0) hd[(size_t)c * N + (size_t)sm] += 0.5 * P[b][c];
                    }
                }
            }
    return E;
}

/* Exported: Delta f at one site for a given director and gradient (tests);
 * G, P are [3][3] row-major with G[3b+c] = d_b n_c. */
double or_frank3_point(const or_params* p, const double* nc, const double* Gflat, double* dfdn, double* Pflat)
{
    double G[3][3], P[3][3];
    for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c) G[b][c] = Gflat[3 * b + c];
    double f = frank3_point(p, nc, G, dfdn, P);
    for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c) Pflat[3 * b + c] = P[b][c];
    return f;
}

/* Exported: the three-constant correction's energy sum and field (tests). */
double or_frank3_field(const or_params* p, const double* n, double* hd) { return frank3_field(p, n, hd); }

/* Strain rate D and vorticity W (Sec. II.A) from du[a][b] = d_a u_b. */
static void strain_vorticity(const double du[3][3], double D[3][3], double W[3][3])
{
    for (int a = 0; a < 3; ++a)
        for (int m = 0; m < 3; ++m) {
            D[a][m] = 0.5 * (du[a][m] + du[m][a]);
            W[a][m] = 0.5 * (du[m][a] - du[a][m]);
        }
}

/* Molecular field of a director field (exported for the energy check). */
void or_molecular_field(const or_params* p, const double* n, double* h_out)
{
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    double* hd = p->frank3 ? (double*)malloc(3 * N * sizeof(double)) : NULL;
    if (hd) frank3_field(p, n, hd);
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t s = site(p, x, y, z);
                double nc[3], dn[3][3], lap[3], du[3][3], h[3];
                n_at(p, n, x, y, z, nc);
                local_derivs(p, n, NULL, x, y, z, dn, lap, du);
                molecular_field(p, n, x, y, z, nc, lap, h);
                for (int a = 0; a < 3; ++a) h_out[(size_t)a * N + s] = h[a] + (hd ? hd[(size_t)a * N + s] : 0.0);
            }
    free(hd);
}

/* Time derivative of the director, Eq. director-time-eq, evaluated for the
 * director field n and the velocity field u:
 *   dn_mu/dt = h_mu/gamma1 - (gamma2/gamma1) n_a D_{a mu} - u_g d_g n_mu + W_{mu g} n_g. */
void or_director_rate(const or_params* p, const double* n, const double* u, double* ndot)
{
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    double* hd = p->frank3 ? (double*)malloc(3 * N * sizeof(double)) : NULL;
    if (hd) frank3_field(p, n, hd);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t s = site(p, x, y, z);
                if (is_solid(p, s)) { /* fixed director */
                    for (int m = 0; m < 3; ++m) ndot[(size_t)m * N + s] = 0.0;
                    continue;
                }
                double nc[3], uc[3], dn[3][3], lap[3], du[3][3], h[3], D[3][3], W[3][3];
                n_at(p, n, x, y, z, nc);
                u_at(p, u, x, y, z, uc);
                local_derivs(p, n, u, x, y, z, dn, lap, du);
                molecular_field(p, n, x, y, z, nc, lap, h);
                if (hd)
                    for (int a = 0; a < 3; ++a) h[a] += hd[(size_t)a * N + s];
                strain_vorticity(du, D, W);
                for (int m = 0; m < 3; ++m) {
                    double r = h[m] / p->gamma1;
                    for (int a = 0; a < 3; ++a) r -= (p->gamma2 / p->gamma1) * nc[a] * D[a][m];
                    for (int g = 0; g < 3; ++g) r -= uc[g] * dn[g][m];
                    for (int g = 0; g < 3; ++g) r += W[m][g] * nc[g];
                    ndot[(size_t)m * N + s] = r;
                }
            }
    free(hd);
}

/* Scale the director at every fluid site to unit length. */
static void normalise(const or_params* p, double* n)
{
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    for (size_t s = 0; s < N; ++s) {
        if (is_solid(p, s)) continue;
        double len = sqrt(n[s] * n[s] + n[N + s] * n[N + s] + n[2 * N + s] * n[2 * N + s]);
        for (int a = 0; a < 3; ++a) n[(size_t)a * N + s] /= len;
    }
}

/* One FD step of length dt_fd with the predictor-corrector scheme of Sec. II.B,
 * followed by renormalisation |n| = 1.  u is held fixed during the step.
 * work must hold 9*N doubles; on return work[0 .. 3N) holds the averaged time
 * derivative (1/2)[(dn/dt)_old + (dn/dt)_P] that advanced n. */
void or_fd_step(const or_params* p, double* n, const double* u, double* work)
{
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    double* ndot_old = work;
    double* nP = work + 3 * N;
    double* ndot_P = work + 6 * N;
    or_director_rate(p, n, u, ndot_old);
    for (size_t k = 0; k < 3 * N; ++k) nP[k] = n[k] + p->dt_fd * ndot_old[k];
    if (p->renorm_predictor) normalise(p, nP);
    or_director_rate(p, nP, u, ndot_P);
    for (size_t k = 0; k < 3 * N; ++k) ndot_old[k] = 0.5 * (ndot_old[k] + ndot_P[k]); /* averaged rate */
    for (size_t k = 0; k < 3 * N; ++k) n[k] = n[k] + p->dt_fd * ndot_old[k];
    for (size_t s = 0; s < N; ++s) {
        if (is_solid(p, s)) continue;
        double len = sqrt(n[s] * n[s] + n[N + s] * n[N + s] + n[2 * N + s] * n[2 * N + s]);
        for (int a = 0; a < 3; ++a) n[(size_t)a * N + s] /= len;
    }
}

/* ---------------------------------------------------------------- stress */

/* Kinematic transport from the director equation, projected normal to n:
 * N = [h_perp - gamma2 (I - n n) D n] / gamma1. */
void or_transport_point(const double* n, const double* h, const double* Dflat, double gamma1, double gamma2,
                        double* Nout)
{
    double hn = h[0] * n[0] + h[1] * n[1] + h[2] * n[2];
    double Dn[3], nDn = 0.0;
    for (int a = 0; a < 3; ++a) {
        Dn[a] = 0.0;
        for (int b = 0; b < 3; ++b) Dn[a] += Dflat[3 * a + b] * n[b];
    }
    for (int a = 0; a < 3; ++a) nDn += n[a] * Dn[a];
    for (int m = 0; m < 3; ++m) {
        double hperp = h[m] - hn * n[m];
        double Dn_perp = Dn[m] - n[m] * nDn;
        Nout[m] = (hperp - gamma2 * Dn_perp) / gamma1;
    }
}

/* Viscous part of the stress in Eq. force-lc-eq (with alpha_4'), for a given
 * director n, strain rate D and kinematic transport N; sigma[3a+b]. */
void or_viscous_stress_point(const or_params* p, const double* n, const double* Dflat, const double* Nv, double* sig)
{
    double Dn[3], nDn = 0.0;
    for (int a = 0; a < 3; ++a) {
        Dn[a] = 0.0;
        for (int m = 0; m < 3; ++m) Dn[a] += n[m] * Dflat[3 * m + a]; /* n_mu D_{mu a} */
    }
    for (int m = 0; m < 3; ++m)
        for (int r = 0; r < 3; ++r) nDn += n[m] * n[r] * Dflat[3 * m + r];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            sig[3 * a + b] = p->alpha1 * n[a] * n[b] * nDn + p->alpha2 * n[b] * Nv[a] + p->alpha3 * n[a] * Nv[b] +
                             p->alpha4p * Dflat[3 * a + b] + p->alpha5 * n[b] * Dn[a] + p->alpha6 * n[a] * Dn[b];
}

/* Elastic (Ericksen) stress for the one-constant chiral energy density
 * f = K/2 d_b n_g d_b n_g + K q0 n . curl n + K q0^2/2:
 * sigma^e_ab = - d_a n_g  df/d(d_b n_g) = - d_a n_g [K d_b n_g + K q0 eps_{c b g} n_c];
 * dn[3*b+g] = d_b n_g. */
void or_elastic_stress_point(const or_params* p, const double* n, const double* dn, double* sig)
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int g = 0; g < 3; ++g) {
                double dfdG = p->K * dn[3 * b + g];
                for (int c = 0; c < 3; ++c) dfdG += p->K * p->q0 * levi(c, b, g) * n[c];
                s -= dn[3 * a + g] * dfdG;
            }
            sig[3 * a + b] = s;
        }
}

/* LC stress tensor at every fluid site: sigma = sigma^v(alpha_4') + sigma^e,
 * from the director n, its molecular field h and the velocity u.  With
 * n_from_rate and a rate field ndot (the corrector's averaged dn/dt) the
 * kinematic transport is N = (I - n n)(ndot + u.grad n - W n) (Sec. II.A,
 * projected normal to n as the director-equation form is);
 * otherwise (or when ndot is NULL) N comes from the director equation. */
void or_stress(const or_params* p, const double* n, const double* u, const double* ndot, double* sigma)
{
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    double* hd = p->frank3 ? (double*)malloc(3 * N * sizeof(double)) : NULL;
    if (hd) frank3_field(p, n, hd);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t s = site(p, x, y, z);
                if (is_solid(p, s)) {
                    for (int k = 0; k < 9; ++k) sigma[(size_t)k * N + s] = 0.0;
                    continue;
                }
                double nc[3], dn[3][3], lap[3], du[3][3], h[3], D[3][3], W[3][3];
                n_at(p, n, x, y, z, nc);
                local_derivs(p, n, u, x, y, z, dn, lap, du);
                molecular_field(p, n, x, y, z, nc, lap, h);
                if (hd)
                    for (int a = 0; a < 3; ++a) h[a] += hd[(size_t)a * N + s];
                strain_vorticity(du, D, W);
                double Dflat[9], dnflat[9], Nv[3], sv[9], se[9];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        Dflat[3 * a + b] = D[a][b];
                        dnflat[3 * a + b] = dn[a][b];
                    }
                if (p->n_from_rate && ndot != NULL) {
                    double t[3], uc[3], nt = 0.0;
                    u_at(p, u, x, y, z, uc);
                    for (int m = 0; m < 3; ++m) {
                        t[m] = ndot[(size_t)m * N + s];
                        for (int g = 0; g < 3; ++g) t[m] += uc[g] * dn[g][m] - W[m][g] * nc[g];
                    }
                    for (int m = 0; m < 3; ++m) nt += nc[m] * t[m];
                    for (int m = 0; m < 3; ++m) Nv[m] = t[m] - nt * nc[m];
                } else {
                    or_transport_point(nc, h, Dflat, p->gamma1, p->gamma2, Nv);
                }
                or_viscous_stress_point(p, nc, Dflat, Nv, sv);
                or_elastic_stress_point(p, nc, dnflat, se);
                if (hd) {
                    /* Ericksen stress of the correction: -d_a n_g dDelta f/d(d_b n_g) */
                    double dfdn[3], P[3][3];
                    frank3_point(p, nc, dn, dfdn, P);
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            for (int g = 0; g < 3; ++g) se[3 * a + b] -= dn[a][g] * P[b][g];
                }
                for (int k = 0; k < 9; ++k) sigma[(size_t)k * N + s] = sv[k] + se[k];
            }
    free(hd);
}

/* F^LC_a = d_b sigma_ab with central differences; sigma = 0 at solid ghosts
 * (ghost_sigma = 1: the stress of the adjacent fluid layer at the plates'
 * ghost layers). */
void or_force(const or_params* p, const double* sigma, double* F)
{
    const size_t N = (size_t)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t s = site(p, x, y, z);
                if (is_solid(p, s)) {
                    for (int a = 0; a < 3; ++a) F[(size_t)a * N + s] = 0.0;
                    continue;
                }
                for (int a = 0; a < 3; ++a) {
                    double div = 0.0;
                    for (int b = 0; b < 3; ++b) {
                        int d[3] = {0, 0, 0};
                        d[b] = 1;
                        const double ghost = p->ghost_sigma ? sigma[(size_t)(3 * a + b) * N + s] : 0.0;
                        double sp = ghost, sm = ghost;
                        int zp = z + d[2], zm = z - d[2];
                        if (!(p->walls_z && (zp < 0 || zp >= p->nz)))
                            sp = sigma[(size_t)(3 * a + b) * N +
                                       site(p, wrap(x + d[0], p->nx), wrap(y + d[1], p->ny), wrap(zp, p->nz))];
                        if (!(p->walls_z && (zm < 0 || zm >= p->nz)))
                            sm = sigma[(size_t)(3 * a + b) * N +
                                       site(p, wrap(x - d[0], p->nx), wrap(y - d[1], p->ny), wrap(zm, p->nz))];
                        div += 0.5 * (sp - sm);
                    }
                    F[(size_t)a * N + s] = div;
                }
            }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
