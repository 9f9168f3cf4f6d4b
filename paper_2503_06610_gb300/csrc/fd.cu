// fd.cu -- finite-difference director update and LC stress / force
// (arXiv:2503.06610, Secs. II.A-II.B, Eq. director-time-eq, Eq. force-lc-eq,
// Eq. free-energy-eq).
//
// Kernels (one thread per site, radius-1 stencils, central differences):
//   fd_predict : (dn/dt)_old from n and u;  n^P = n + dt_FD (dn/dt)_old
//   fd_correct : (dn/dt)_P from n^P and u;  n <- n + dt_FD/2 [(dn/dt)_old + (dn/dt)_P],
//                then n <- n/|n|  (in place: each site reads only its own n)
//   stress     : sigma = sigma^v(alpha_4') + sigma^e from the new n and u
//   force      : F_lc,a = d_b sigma_ab, zero stress at solid ghost layers
// The molecular field is the one-constant chiral form
//   h = K lap n - 2 K q0 curl n + W0 n_z z_hat
// (compact Laplacian, central curl), the exact -dE/dn of the lattice energy
// (a sum over nearest-neighbour links).  Beyond the plates the ghost velocity
// is zero and the ghost director is z_hat (homeotropic) or the adjacent layer.
// A plate without anchoring is a free surface: its links carry no energy, so
// on the two plate layers the chiral term lacks the link to the ghost layer,
// which the central curl over the copied ghost would contribute; the kernels
// take that link out again (free_plate_side).
#include "diag_sum.cuh"

namespace nh {

namespace {

template <typename Real>
__device__ __forceinline__ void site_xyz(const Geom& g, int s, int& x, int& y, int& z)
{
    x = s % g.nx;
    const int t = s / g.nx;
    y = t % g.ny;
    z = t / g.ny;
}

// Director at (x, y, z) with x, y already wrapped; z may be -1 or nz.
template <typename Real>
__device__ __forceinline__ void dir_at(const Real* __restrict__ n, const Geom& g, int x, int y, int z, Real out[3])
{
    if (g.walls) {
        if (z < 0 || z >= g.nz) {
            if (g.anchoring == NH_ANCHOR_HOMEOTROPIC) {
                out[0] = Real(0);
                out[1] = Real(0);
                out[2] = Real(1);
                return;
            }
            z = z < 0 ? 0 : g.nz - 1;
        }
    } else {
        z = wrap_p(z, g.nz);
    }
    const int s = x + g.nx * (y + g.ny * z);
    out[0] = n[s];
    out[1] = n[g.N + s];
    out[2] = n[2 * g.N + s];
}

template <typename Real>
__device__ __forceinline__ void vel_at(const Real* __restrict__ u, const Geom& g, int x, int y, int z, Real out[3],
                                       const unsigned char* solid = nullptr)
{
    if (g.walls) {
        if (z < 0 || z >= g.nz) {
            out[0] = out[1] = out[2] = Real(0);
            return;
        }
    } else {
        z = wrap_p(z, g.nz);
    }
    const int s = x + g.nx * (y + g.ny * z);
    if (solid != nullptr && solid[s]) {  // obstacle: no-slip
        out[0] = out[1] = out[2] = Real(0);
        return;
    }
    out[0] = u[s];
    out[1] = u[g.N + s];
    out[2] = u[2 * g.N + s];
}

// Sum over the six sites at distance 2 along the axes, S2[c] = sum_b
// n_c(x + 2 e_b) + n_c(x - 2 e_b), with the ghost rule of dir_at beyond the
// plates (reading flag lap_wide: the second derivative of the molecular field
// as the central difference of the central difference,
// (S2 - 6 n)/4 = sum_b [n(x + 2e_b) - 2 n(x) + n(x - 2e_b)]/4).
template <typename Real>
__device__ __forceinline__ void wide_sum(const Real* __restrict__ n, const Geom& g, int x, int y, int z, Real S2[3])
{
    auto wrapf = [](int a, int m) {
        a %= m;
        return a < 0 ? a + m : a;
    };
    Real v[6][3];
    dir_at(n, g, wrapf(x + 2, g.nx), y, z, v[0]);
    dir_at(n, g, wrapf(x - 2, g.nx), y, z, v[1]);
    dir_at(n, g, x, wrapf(y + 2, g.ny), z, v[2]);
    dir_at(n, g, x, wrapf(y - 2, g.ny), z, v[3]);
    const int zp = g.walls ? z + 2 : wrapf(z + 2, g.nz), zm = g.walls ? z - 2 : wrapf(z - 2, g.nz);
    dir_at(n, g, x, y, zp, v[4]);
    dir_at(n, g, x, y, zm, v[5]);
#pragma unroll
    for (int c = 0; c < 3; ++c) S2[c] = ((v[0][c] + v[1][c]) + (v[2][c] + v[3][c])) + (v[4][c] + v[5][c]);
}

// Plate layer of a channel whose plates have no anchoring: -1 on the lowest
// layer, +1 on the highest, 0 elsewhere (and 0 when nz = 1, where both apply
// and cancel).  The central curl over the copied ghost layer there holds the
// term of a link that carries no energy; removing it adds
//   dh = side K q0 (-n_y, n_x, 0)
// to the molecular field (-K q0 z x n below, +K q0 z x n above).
__device__ __forceinline__ int free_plate_side(const Geom& g, int z)
{
    if (!g.walls || g.anchoring != NH_ANCHOR_NONE) return 0;
    return (z == g.nz - 1 ? 1 : 0) - (z == 0 ? 1 : 0);
}

// 7-point neighbourhood: index 0 = centre, 1 + 2b = +e_b, 2 + 2b = -e_b.
template <typename Real>
__device__ __forceinline__ void gather7(const Real* __restrict__ f, const Geom& g, int x, int y, int z, Real v[7][3],
                                        bool director, const unsigned char* solid = nullptr)
{
    const int xp = wrap_p(x + 1, g.nx), xm = wrap_p(x - 1, g.nx);
    const int yp = wrap_p(y + 1, g.ny), ym = wrap_p(y - 1, g.ny);
    if (director) {
        dir_at(f, g, x, y, z, v[0]);
        dir_at(f, g, xp, y, z, v[1]);
        dir_at(f, g, xm, y, z, v[2]);
        dir_at(f, g, x, yp, z, v[3]);
        dir_at(f, g, x, ym, z, v[4]);
        dir_at(f, g, x, y, z + 1, v[5]);
        dir_at(f, g, x, y, z - 1, v[6]);
    } else {
        vel_at(f, g, x, y, z, v[0], solid);
        vel_at(f, g, xp, y, z, v[1], solid);
        vel_at(f, g, xm, y, z, v[2], solid);
        vel_at(f, g, x, yp, z, v[3], solid);
        vel_at(f, g, x, ym, z, v[4], solid);
        vel_at(f, g, x, y, z + 1, v[5], solid);
        vel_at(f, g, x, y, z - 1, v[6], solid);
    }
}

// Differences and sums of a 7-point neighbourhood: e[b][c] = n_c(+e_b) -
// n_c(-e_b) (twice the central derivative d_b n_c), v[b][c] the same for u,
// S[c] = sum of the six neighbours of n_c (compact Laplacian = S - 6 n_c) and
// ce = curl of e (twice the central curl of n).
template <typename Real>
__device__ __forceinline__ void stencil_diffs(const Real nn[7][3], const Real uu[7][3], Real e[3][3], Real v[3][3],
                                              Real S[3], Real ce[3])
{
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            e[b][c] = nn[1 + 2 * b][c] - nn[2 + 2 * b][c];
            v[b][c] = uu[1 + 2 * b][c] - uu[2 + 2 * b][c];
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) S[c] = ((nn[1][c] + nn[2][c]) + (nn[3][c] + nn[4][c])) + (nn[5][c] + nn[6][c]);
    ce[0] = e[1][2] - e[2][1];
    ce[1] = e[2][0] - e[0][2];
    ce[2] = e[0][1] - e[1][0];
}

// Eq. director-time-eq: dn_m/dt = h_m/g1 - (g2/g1) n_a D_am - u_a d_a n_m + W_ma n_a,
// with h = K lap n - 2 K q0 curl n + W0 n_z z_hat, D = (du + du^T)/2 and
// W_ma = (d_a u_m - d_m u_a)/2.  In the differences above (lambda = g2/g1):
//   h_m/g1 = kg (S_m - 6 n_m) - kqg ce_m + w0g n_z delta_mz,
//   -lambda n_a D_am + W_ma n_a = sum_a n_a [(1 - lambda)/4 v[a][m] - (1 + lambda)/4 v[m][a]],
//   -u_a d_a n_m = -1/2 sum_a u_a e[a][m].
// hx (optional) is an extra molecular field (three-constant correction);
// side is free_plate_side() of the point's layer; S2 (optional, lap_wide) the
// distance-2 sum of wide_sum, which replaces the compact Laplacian.
template <typename Real>
__device__ __forceinline__ void director_rate(const Real nn[7][3], const Real uu[7][3], const FDPar<Real>& p,
                                              Real rate[3], const Real* hx = nullptr, int side = 0,
                                              const Real* S2 = nullptr)
{
    Real e[3][3], v[3][3], S[3], ce[3];
    stencil_diffs(nn, uu, e, v, S, ce);
    const Real* n = nn[0];
    Real w1[3], w2[3], hu[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w1[a] = p.c1 * n[a];
        w2[a] = p.c2 * n[a];
        hu[a] = Real(-0.5) * uu[0][a];
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        Real r = S2 != nullptr ? Real(0.25) * p.kg * (S2[m] - Real(6) * n[m]) : p.kg * (S[m] - Real(6) * n[m]);
        r = fma(-p.kqg, ce[m], r);
        if (m == 2) r = fma(p.w0g, n[2], r);
        if (hx != nullptr) r = fma(hx[m], p.inv_gamma1, r);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            r = fma(v[a][m], w1[a], r);
            r = fma(v[m][a], w2[a], r);
            r = fma(hu[a], e[a][m], r);
        }
        rate[m] = r;
    }
    if (side != 0) {
        const Real sk = Real(side) * p.kqg;
        rate[0] = fma(-sk, n[1], rate[0]);
        rate[1] = fma(sk, n[0], rate[1]);
    }
}

// ---- three-constant correction (per-site path)
//
// Stage P: P[b][c] = d df/d(d_b n_c) of the correction at every site, from the
// central gradient of the field m (n or n^P).  The field of the correction at
// site y is the exact -d(sum df)/dn_c(y):
//   hx_c(y) = -d df/d n_c(y) + 1/2 sum_b [P_bc(y + e_b) - P_bc(y - e_b)]
// with P = 0 at ghost sites; without anchoring the ghost layer copies the
// adjacent fluid layer, which adds +P_zc(y)/2 on the lowest and -P_zc(y)/2 on
// the highest layer.
template <typename Real>
__device__ __forceinline__ void frank3_p_site(const FDChan<Real>& c, const Real* m, int s)
{
    if (c.solid != nullptr && c.solid[s]) {  // no energy at obstacle nodes
#pragma unroll
        for (int k = 0; k < 9; ++k) c.P3[k * c.g.N + s] = Real(0);
        return;
    }
    int x, y, z;
    site_xyz<Real>(c.g, s, x, y, z);
    Real nn[7][3];
    gather7(m, c.g, x, y, z, nn, true);
    Real G[3][3], dfdn[3], P[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int k = 0; k < 3; ++k) G[b][k] = Real(0.5) * (nn[1 + 2 * b][k] - nn[2 + 2 * b][k]);
    frank3_site(nn[0], G, c.p.kd1, c.p.kd2, c.p.kd3, c.p.q0, dfdn, P);
    const int N = c.g.N;
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int k = 0; k < 3; ++k) c.P3[(3 * b + k) * N + s] = P[b][k];
}

template <typename Real>
__device__ __forceinline__ void frank3_field_site(const FDChan<Real>& c, const Real nn[7][3], int x, int y, int z,
                                                  Real hx[3])
{
    const Geom& g = c.g;
    const int N = g.N;
    Real G[3][3], dfdn[3], P[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int k = 0; k < 3; ++k) G[b][k] = Real(0.5) * (nn[1 + 2 * b][k] - nn[2 + 2 * b][k]);
    frank3_site(nn[0], G, c.p.kd1, c.p.kd2, c.p.kd3, c.p.q0, dfdn, P);
#pragma unroll
    for (int k = 0; k < 3; ++k) hx[k] = -dfdn[k];
    const int xp = wrap_p(x + 1, g.nx), xm = wrap_p(x - 1, g.nx);
    const int yp = wrap_p(y + 1, g.ny), ym = wrap_p(y - 1, g.ny);
    const int row = g.nx * (y + g.ny * z);
    const int sxp = xp + row, sxm = xm + row;
    const int syp = x + g.nx * (yp + g.ny * z), sym = x + g.nx * (ym + g.ny * z);
    int zp = z + 1, zm = z - 1;
    bool zp_ok = true, zm_ok = true;
    if (g.walls) {
        zp_ok = zp < g.nz;
        zm_ok = zm >= 0;
    } else {
        zp = wrap_p(zp, g.nz);
        zm = wrap_p(zm, g.nz);
    }
    const int szp = x + g.nx * (y + g.ny * (zp_ok ? zp : 0)), szm = x + g.nx * (y + g.ny * (zm_ok ? zm : 0));
    const Real* P3 = c.P3;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Real acc = P3[(0 + k) * N + sxp] - P3[(0 + k) * N + sxm];
        acc += P3[(3 + k) * N + syp] - P3[(3 + k) * N + sym];
        if (zp_ok) acc += P3[(6 + k) * N + szp];
        if (zm_ok) acc -= P3[(6 + k) * N + szm];
        if (g.walls && g.anchoring != NH_ANCHOR_HOMEOTROPIC) {
            if (z == 0) acc += P[2][k];
            if (z == g.nz - 1) acc -= P[2][k];
        }
        hx[k] += Real(0.5) * acc;
    }
}

template <typename Real>
__device__ __forceinline__ void fd_predict_site(const FDChan<Real>& c, int s)
{
    const int N = c.g.N;
    if (c.solid != nullptr && c.solid[s]) {  // obstacle: the director is held
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            c.ndot[a * N + s] = Real(0);
            c.nP[a * N + s] = c.n[a * N + s];
        }
        return;
    }
    int x, y, z;
    site_xyz<Real>(c.g, s, x, y, z);
    Real nn[7][3], uu[7][3], r[3];
    gather7(c.n, c.g, x, y, z, nn, true);
    gather7(c.u, c.g, x, y, z, uu, false, c.solid);
    const int side = free_plate_side(c.g, z);
    Real S2[3];
    if (c.p.lap_wide) wide_sum(c.n, c.g, x, y, z, S2);
    const Real* s2 = c.p.lap_wide ? S2 : nullptr;
    if (c.P3 != nullptr) {
        Real hx[3];
        frank3_field_site(c, nn, x, y, z, hx);
        director_rate(nn, uu, c.p, r, hx, side, s2);
    } else {
        director_rate(nn, uu, c.p, r, (const Real*)nullptr, side, s2);
    }
    Real np[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) np[a] = nn[0][a] + c.p.dt * r[a];
    if (c.p.renorm_p) {
        const Real inv = Real(1) / sqrt(np[0] * np[0] + np[1] * np[1] + np[2] * np[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) np[a] *= inv;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        c.ndot[a * N + s] = r[a];
        c.nP[a * N + s] = np[a];
    }
}

template <typename Real>
__device__ __forceinline__ void fd_correct_site(const FDChan<Real>& c, int s)
{
    if (c.solid != nullptr && c.solid[s]) return;  // obstacle: the director is held
    int x, y, z;
    site_xyz<Real>(c.g, s, x, y, z);
    Real nn[7][3], uu[7][3], r[3];
    gather7(c.nP, c.g, x, y, z, nn, true);
    gather7(c.u, c.g, x, y, z, uu, false, c.solid);
    const int side = free_plate_side(c.g, z);
    Real S2[3];
    if (c.p.lap_wide) wide_sum(c.nP, c.g, x, y, z, S2);
    const Real* s2 = c.p.lap_wide ? S2 : nullptr;
    if (c.P3 != nullptr) {
        Real hx[3];
        frank3_field_site(c, nn, x, y, z, hx);
        director_rate(nn, uu, c.p, r, hx, side, s2);
    } else {
        director_rate(nn, uu, c.p, r, (const Real*)nullptr, side, s2);
    }
    const int N = c.g.N;
    Real nw[3], avg[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        avg[a] = Real(0.5) * (c.ndot[a * N + s] + r[a]);
        nw[a] = c.n[a * N + s] + c.p.dt * avg[a];
    }
    if (c.p.n_rate) {  // the averaged rate stays in ndot for the stress (reading flag n_from_rate)
#pragma unroll
        for (int a = 0; a < 3; ++a) c.ndot[a * N + s] = avg[a];
    }
    const Real inv = Real(1) / sqrt(nw[0] * nw[0] + nw[1] * nw[1] + nw[2] * nw[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) c.n[a * N + s] = nw[a] * inv;
}

// LC stress (Eq. force-lc-eq, bracket) at one point from its 7-point
// neighbourhood of n and u: sigma[3a+b].
// S2 (optional, lap_wide): the distance-2 sum of wide_sum; rate (optional,
// n_from_rate): the corrector's averaged dn/dt at the point, from which
// N = P_perp(rate) + u.grad n - W n replaces the director-equation form.
template <typename Real>
__device__ __forceinline__ void stress_point(const Real nn[7][3], const Real uu[7][3], const FDPar<Real>& p,
                                             Real sig[9], const Real* hx = nullptr, const Real* Pd = nullptr,
                                             int side = 0, const Real* S2 = nullptr, const Real* rate = nullptr)
{
    // In the differences of stencil_diffs (Ds = v + v^T = 4 D, Dn_a = Ds_am n_m = 4 D_am n_m):
    //   N_m = [h_m - (h.n) n_m]/g1 - lambda/4 [Dn_m - (n.Dn) n_m]       (kinematic transport, normal to n)
    //   sigma^v_ab = n_b P_a + n_a Q_b + a4'/4 Ds_ab,
    //     P_a = a1/4 (n.Dn) n_a + a2 N_a + a5/4 Dn_a,   Q_b = a3 N_b + a6/4 Dn_b,
    //   sigma^e_ab = -d_a n_g df/d(d_b n_g) = -K/4 e_a.e_b - K q0/2 (e_a x n)_b
    //     (one-constant chiral density; e_a = row a of e), minus 1/2 e_ag Pd_bg for the
    //     three-constant correction Pd = d(Delta f)/d(d n).
    Real e[3][3], v[3][3], S[3], ce[3];
    stencil_diffs(nn, uu, e, v, S, ce);
    const Real* n = nn[0];
    Real h[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const Real lap = S2 != nullptr ? Real(0.25) * (S2[m] - Real(6) * n[m]) : S[m] - Real(6) * n[m];
        h[m] = fma(-p.kq, ce[m], p.K * lap);
        if (hx != nullptr) h[m] += hx[m];
    }
    h[2] = fma(p.W0, n[2], h[2]);
    if (side != 0) {  // free plate layer (see free_plate_side)
        const Real sk = Real(side) * p.kq;
        h[0] = fma(-sk, n[1], h[0]);
        h[1] = fma(sk, n[0], h[1]);
    }
    Real Ds[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) {
            Ds[a][b] = v[a][b] + v[b][a];
            Ds[b][a] = Ds[a][b];
        }
    Real Dn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Dn[a] = fma(Ds[a][2], n[2], fma(Ds[a][1], n[1], Ds[a][0] * n[0]));
    const Real nDn = fma(n[2], Dn[2], fma(n[1], Dn[1], n[0] * Dn[0]));
    const Real hn = fma(n[2], h[2], fma(n[1], h[1], n[0] * h[0]));
    Real P[3], Q[3];
    Real Nr[3] = {0, 0, 0};
    if (rate != nullptr) {
        // t_m = rate_m + u_a d_a n_m - W_ma n_a, W_ma = (d_a u_m - d_m u_a)/2 (in the raw
        // differences u_a e[a][m]/2 and (v[a][m] - v[m][a]) n_a / 4); N = t - (n.t) n
        Real t[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            Real acc = rate[m];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                acc = fma(Real(0.5) * uu[0][a], e[a][m], acc);
                acc = fma(Real(-0.25) * (v[a][m] - v[m][a]), n[a], acc);
            }
            t[m] = acc;
        }
        const Real nt = fma(n[2], t[2], fma(n[1], t[1], n[0] * t[0]));
#pragma unroll
        for (int m = 0; m < 3; ++m) Nr[m] = fma(-nt, n[m], t[m]);
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const Real Nm = rate != nullptr ? Nr[m]
                                        : p.inv_gamma1 * fma(-hn, n[m], h[m]) - p.g2q * fma(-nDn, n[m], Dn[m]);
        P[m] = fma(p.a5q, Dn[m], fma(p.a2, Nm, p.a1q * nDn * n[m]));
        Q[m] = fma(p.a6q, Dn[m], p.a3 * Nm);
    }
    Real G[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) {
            G[a][b] = fma(e[a][2], e[b][2], fma(e[a][1], e[b][1], e[a][0] * e[b][0]));
            G[b][a] = G[a][b];
        }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const Real X[3] = {e[a][1] * n[2] - e[a][2] * n[1], e[a][2] * n[0] - e[a][0] * n[2],
                           e[a][0] * n[1] - e[a][1] * n[0]};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            Real s = n[b] * P[a];
            s = fma(n[a], Q[b], s);
            s = fma(p.a4q, Ds[a][b], s);
            s = fma(-p.k4, G[a][b], s);
            s = fma(-p.kq2, X[b], s);
            if (Pd != nullptr) {
#pragma unroll
                for (int g = 0; g < 3; ++g) s = fma(Real(-0.5) * e[a][g], Pd[3 * b + g], s);
            }
            sig[3 * a + b] = s;
        }
    }
}

template <typename Real>
__device__ __forceinline__ void stress_site(const FDChan<Real>& c, int s)
{
    if (c.solid != nullptr && c.solid[s]) {  // zero stress at obstacle nodes
#pragma unroll
        for (int k = 0; k < 9; ++k) c.sigma[k * c.g.N + s] = Real(0);
        return;
    }
    int x, y, z;
    site_xyz<Real>(c.g, s, x, y, z);
    Real nn[7][3], uu[7][3], sig[9];
    gather7(c.n, c.g, x, y, z, nn, true);
    gather7(c.u, c.g, x, y, z, uu, false, c.solid);
    Real S2[3], rate[3];
    if (c.p.lap_wide) wide_sum(c.n, c.g, x, y, z, S2);
    if (c.p.n_rate) {
#pragma unroll
        for (int a = 0; a < 3; ++a) rate[a] = c.ndot[a * c.g.N + s];
    }
    const Real* s2 = c.p.lap_wide ? S2 : nullptr;
    const Real* rt = c.p.n_rate ? rate : nullptr;
    if (c.P3 != nullptr) {
        Real hx[3], Pd[9];
        frank3_field_site(c, nn, x, y, z, hx);
#pragma unroll
        for (int k = 0; k < 9; ++k) Pd[k] = c.P3[k * c.g.N + s];
        stress_point(nn, uu, c.p, sig, hx, Pd, free_plate_side(c.g, z), s2, rt);
    } else {
        stress_point(nn, uu, c.p, sig, (const Real*)nullptr, (const Real*)nullptr, free_plate_side(c.g, z), s2, rt);
    }
    const int N = c.g.N;
#pragma unroll
    for (int k = 0; k < 9; ++k) c.sigma[k * N + s] = sig[k];
}

template <typename Real>
__device__ __forceinline__ void force_site(const FDChan<Real>& c, int s)
{
    const Geom& g = c.g;
    const int N = g.N;
    if (c.solid != nullptr && c.solid[s]) {  // no force on obstacle nodes
#pragma unroll
        for (int a = 0; a < 3; ++a) c.F[a * N + s] = Real(0);
        return;
    }
    int x, y, z;
    site_xyz<Real>(c.g, s, x, y, z);
    const int xp = wrap_p(x + 1, g.nx), xm = wrap_p(x - 1, g.nx);
    const int yp = wrap_p(y + 1, g.ny), ym = wrap_p(y - 1, g.ny);
    int zp = z + 1, zm = z - 1;
    bool zp_ok = true, zm_ok = true;
    if (g.walls) {
        zp_ok = zp < g.nz;
        zm_ok = zm >= 0;
    } else {
        zp = wrap_p(zp, g.nz);
        zm = wrap_p(zm, g.nz);
    }
    const int sxp = xp + g.nx * (y + g.ny * z), sxm = xm + g.nx * (y + g.ny * z);
    const int syp = x + g.nx * (yp + g.ny * z), sym = x + g.nx * (ym + g.ny * z);
    const int szp = x + g.nx * (y + g.ny * (zp_ok ? zp : 0)), szm = x + g.nx * (y + g.ny * (zm_ok ? zm : 0));
    // ghost stress beyond a plate: zero, or the wall layer's own (mirror)
    const Real gmir = c.p.mirror ? Real(1) : Real(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const Real* sx = c.sigma + (3 * a + 0) * N;
        const Real* sy = c.sigma + (3 * a + 1) * N;
        const Real* sz = c.sigma + (3 * a + 2) * N;
        const Real dz = (zp_ok ? sz[szp] : gmir * sz[s]) - (zm_ok ? sz[szm] : gmir * sz[s]);
        c.F[a * N + s] = Real(0.5) * ((sx[sxp] - sx[sxm]) + (sy[syp] - sy[sym]) + dz);
    }
}

template <typename Real, int Stage>
__device__ __forceinline__ void fd_stage_site(const FDChan<Real>& c, int s)
{
    if (Stage == 0)
        fd_predict_site(c, s);
    else if (Stage == 1)
        fd_correct_site(c, s);
    else if (Stage == 2)
        stress_site(c, s);
    else if (Stage == 3)
        force_site(c, s);
    else if (Stage == 4) {
        if (c.P3 != nullptr) frank3_p_site(c, c.n, s);  // a batch may mix one- and three-constant channels
    } else {
        if (c.P3 != nullptr) frank3_p_site(c, c.nP, s);
    }
}

template <typename Real, int Stage>
__global__ void __launch_bounds__(256) fd_kernel(const FDChan<Real> c)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < c.g.N) fd_stage_site<Real, Stage>(c, s);
}

// Batched FD stage: a persistent grid walks the (channel, tile) work list.
template <typename Real, int Stage>
__global__ void __launch_bounds__(256) fd_batch_kernel(const FDBatch<Real> b)
{
    const int total = b.prefix[b.count];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int lo = 0, hi = b.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.prefix[mid] <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int s = (t - b.prefix[lo]) * blockDim.x + threadIdx.x;
        if (s < b.ch[lo].g.N) fd_stage_site<Real, Stage>(b.ch[lo], s);
    }
}

// ------------------------------------------------------------------ fused 2.5D kernels
//
// A block owns a tile of kTX x kTY columns and marches up a chunk of kZC (or fewer, fused_zchunk)
// layers.  Planes of n and u with a 2-site halo in x and y sit in a ring of
// three shared-memory slots; the predictor (kernel A) or the stress (kernel
// B) is evaluated on each plane with a 1-site halo, so every stencil reads
// shared memory at fixed offsets and the ghost layers are resolved once, at
// load time.  Kernel A keeps the predicted planes in a ring of three slots;
// kernel B keeps sigma_.x and sigma_.y of two planes.  What only a thread's
// own point needs (u one layer below, the predictor's rate, sigma_.z) stays in
// that thread's registers.
//   kernel A: n, u -> n_new   (predictor, corrector, renormalisation)
//   kernel B: n_new, u -> F   (stress, divergence; sigma never leaves the SM)

constexpr int kTX = 32, kTY = 8, kZC = 16;

// Layers per chunk: kZC, fewer when the channel has too few tiles to fill the
// GPU (a small channel would otherwise run on a handful of blocks): aim at two
// blocks per SM of GB300's 152, down to one layer per chunk (each chunk also
// evaluates the predictor or the stress on the layer below and above it).
// A batch fills the GPU with all its channels' tiles, so its chunk length is
// chosen once from their total (FDChan::zch).
constexpr int kFusedTargetBlocks = 2 * 152;
__host__ __device__ __forceinline__ int fused_xy_tiles(const Geom& g)
{
    return ((g.nx + kTX - 1) / kTX) * ((g.ny + kTY - 1) / kTY);
}
__host__ __device__ __forceinline__ int zchunk_for(long long tile_layers)
{
    const long long c = tile_layers / kFusedTargetBlocks;
    return c < 1 ? 1 : (c > kZC ? kZC : (int)c);
}
template <typename Real>
__host__ __device__ __forceinline__ int fused_zchunk(const FDChan<Real>& c)
{
    return c.zch > 0 ? c.zch : zchunk_for((long long)c.g.nz * fused_xy_tiles(c.g));
}
constexpr int kHX2 = kTX + 4, kHY2 = kTY + 4, kP2 = kHX2 * kHY2;  // plane with a 2-site halo
constexpr int kHX1 = kTX + 2, kHY1 = kTY + 2, kP1 = kHX1 * kHY1;  // plane with a 1-site halo
constexpr int kFusedThreads = 256;

__device__ __forceinline__ int wrapm(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}
__device__ __forceinline__ int slot3(int p) { return ((p % 3) + 3) % 3; }

// Obstacle masks of the three input planes (kP2 bytes each) follow the Real
// arrays; only the kernels of channels with obstacles use them.
constexpr int kMaskBytes = (3 * kP2 + 15) / 16 * 16;
template <typename Real>
size_t fused_a_smem() { return (size_t)(3 * 6 * kP2 + 3 * 4 * kP1) * sizeof(Real) + kMaskBytes; }
template <typename Real>
size_t fused_b_smem() { return (size_t)(3 * 6 * kP2 + 2 * 8 * kP1) * sizeof(Real) + kMaskBytes; }

// Each thread owns at most kPts points of a P2 plane (indices threadIdx.x +
// k * blockDim.x); their wrapped x-y site offsets are computed once per tile.
constexpr int kPts = (kP2 + kFusedThreads - 1) / kFusedThreads;

struct PlaneMap {
    int off[kPts];  // x + nx * y of the point, or -1 if the thread owns no such point
};

__device__ __forceinline__ PlaneMap plane_map(const Geom& g, int x0, int y0)
{
    PlaneMap m;
#pragma unroll
    for (int k = 0; k < kPts; ++k) {
        const int i = threadIdx.x + k * blockDim.x;
        if (i < kP2) {
            const int hx = i % kHX2, hy = i / kHX2;
            m.off[k] = wrapm(x0 - 2 + hx, g.nx) + g.nx * wrapm(y0 - 2 + hy, g.ny);
        } else {
            m.off[k] = -1;
        }
    }
    return m;
}

// Plane zp of n (ghost reading) and u (zero beyond the plates), fetched into
// registers: v[k][0..2] = n, v[k][3..5] = u of the thread's k-th point.  With
// obstacles (Solid) also the mask of each point, sv[k], and u = 0 at solid
// nodes (no-slip); ghost planes hold no solid nodes.
template <typename Real, bool Solid = false>
__device__ __forceinline__ void prefetch_plane(const Real* __restrict__ n, const Real* __restrict__ u, const Geom& g,
                                               const PlaneMap& m, int zp, Real v[kPts][6],
                                               const unsigned char* __restrict__ solid = nullptr,
                                               unsigned char* sv = nullptr)
{
    bool ghost = false;
    int zz;
    if (g.walls) {
        ghost = zp < 0 || zp >= g.nz;
        zz = zp < 0 ? 0 : (zp >= g.nz ? g.nz - 1 : zp);
    } else {
        zz = wrapm(zp, g.nz);
    }
    const bool fixed_dir = ghost && g.anchoring == NH_ANCHOR_HOMEOTROPIC;
    const int N = g.N;  // 3 N < 2^31: 32-bit offsets
    const size_t zoff = (size_t)g.nx * g.ny * zz;
    const Real* __restrict__ nz = n + zoff;
    const Real* __restrict__ uz = u + zoff;
#pragma unroll
    for (int k = 0; k < kPts; ++k) {
        if (m.off[k] < 0) continue;
        const int s = m.off[k];
        bool sol = false;
        if constexpr (Solid) {
            sol = !ghost && solid != nullptr && solid[zoff + s] != 0;  // a batch may mix masked and unmasked channels
            sv[k] = sol ? 1 : 0;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            v[k][a] = fixed_dir ? Real(a == 2 ? 1 : 0) : nz[a * N + s];
            v[k][3 + a] = (ghost || sol) ? Real(0) : uz[a * N + s];
        }
    }
}

// Shared-memory layout of an input plane slot (6 kP2 Reals): the six values
// (n, u) of a point are read with two vector loads in FP32, (n0 n1 n2 u0) as
// float4 [kP2] followed by (u1 u2) as float2 [kP2]; in FP64 as three double2
// arrays (n0 n1), (n2 u0), (u1 u2).
__device__ __forceinline__ void ld_pt(const float* slot, int i, float v[6])
{
    const float4 a = reinterpret_cast<const float4*>(slot)[i];
    const float2 b = reinterpret_cast<const float2*>(slot + 4 * kP2)[i];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y;
}
__device__ __forceinline__ void st_pt(float* slot, int i, const float v[6])
{
    reinterpret_cast<float4*>(slot)[i] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float2*>(slot + 4 * kP2)[i] = make_float2(v[4], v[5]);
}
__device__ __forceinline__ void ld_pt(const double* slot, int i, double v[6])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double2 a = reinterpret_cast<const double2*>(slot + 2 * k * kP2)[i];
        v[2 * k] = a.x;
        v[2 * k + 1] = a.y;
    }
}
__device__ __forceinline__ void st_pt(double* slot, int i, const double v[6])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) reinterpret_cast<double2*>(slot + 2 * k * kP2)[i] = make_double2(v[2 * k], v[2 * k + 1]);
}

// The director alone of point i of an input plane slot: one vector load in
// FP32 (the float4 holds n0 n1 n2 u0), two in FP64.
__device__ __forceinline__ void ld_n(const float* slot, int i, float n[3])
{
    const float4 a = reinterpret_cast<const float4*>(slot)[i];
    n[0] = a.x;
    n[1] = a.y;
    n[2] = a.z;
}
__device__ __forceinline__ void ld_n(const double* slot, int i, double n[3])
{
    const double2 a = reinterpret_cast<const double2*>(slot)[i];
    n[0] = a.x;
    n[1] = a.y;
    n[2] = reinterpret_cast<const double2*>(slot + 2 * kP2)[i].x;
}

// Predictor ring slot (4 kP1 Reals): n^P of a point as one float4 (n0 n1 n2 -)
// in FP32, as three planes of kP1 doubles in FP64.
__device__ __forceinline__ void ld3(const float* slot, int i, float v[3])
{
    const float4 a = reinterpret_cast<const float4*>(slot)[i];
    v[0] = a.x; v[1] = a.y; v[2] = a.z;
}
__device__ __forceinline__ void st3(float* slot, int i, const float v[3])
{
    reinterpret_cast<float4*>(slot)[i] = make_float4(v[0], v[1], v[2], 0.f);
}
__device__ __forceinline__ void ld3(const double* slot, int i, double v[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = slot[a * kP1 + i];
}
__device__ __forceinline__ void st3(double* slot, int i, const double v[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) slot[a * kP1 + i] = v[a];
}

template <typename Real, bool Solid = false>
__device__ __forceinline__ void commit_plane(const PlaneMap& m, const Real v[kPts][6], Real* slot,
                                             const unsigned char* sv = nullptr, unsigned char* mslot = nullptr)
{
#pragma unroll
    for (int k = 0; k < kPts; ++k) {
        if (m.off[k] < 0) continue;
        st_pt(slot, threadIdx.x + k * blockDim.x, v[k]);
        if constexpr (Solid) mslot[threadIdx.x + k * blockDim.x] = sv[k];
    }
}

template <typename Real>
__device__ __forceinline__ void split_pt(const Real* slot, int i, Real n[3], Real u[3])
{
    Real v[6];
    ld_pt(slot, i, v);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        n[a] = v[a];
        u[a] = v[3 + a];
    }
}

// 7-point neighbourhoods of n and u around P2 index i2 of the middle plane.
template <typename Real>
__device__ __forceinline__ void gather_slots(const Real* lo, const Real* mid, const Real* hi, int i2, Real nn[7][3],
                                             Real uu[7][3])
{
    split_pt(mid, i2, nn[0], uu[0]);
    split_pt(mid, i2 + 1, nn[1], uu[1]);
    split_pt(mid, i2 - 1, nn[2], uu[2]);
    split_pt(mid, i2 + kHX2, nn[3], uu[3]);
    split_pt(mid, i2 - kHX2, nn[4], uu[4]);
    split_pt(hi, i2, nn[5], uu[5]);
    split_pt(lo, i2, nn[6], uu[6]);
}

__device__ __forceinline__ bool is_ghost_plane(const Geom& g, int p) { return g.walls && (p < 0 || p >= g.nz); }

// The kP1 points of a 1-halo plane, the tile's own points first: t < kTX kTY
// is the point of thread t (column t % kTX, row t / kTX; a warp reads one row,
// contiguous in shared memory), so the value computed there stays in that
// thread's registers; then the two halo rows and the two halo columns.
constexpr int kOwn = kTX * kTY;
static_assert(kFusedThreads == kOwn, "the fused kernels run one thread per own tile point");
__device__ __forceinline__ void p1_point(int t, int& hx1, int& hy1)
{
    if (t < kOwn) {
        hx1 = t % kTX + 1;
        hy1 = t / kTX + 1;
        return;
    }
    const int e = t - kOwn;
    if (e < 2 * kHX1) {
        hy1 = e < kHX1 ? 0 : kHY1 - 1;
        hx1 = e < kHX1 ? e : e - kHX1;
    } else {
        const int j = e - 2 * kHX1;
        hy1 = 1 + (j >> 1);
        hx1 = (j & 1) ? kHX1 - 1 : 0;
    }
}

// The point of a 1-halo plane that a thread evaluates besides its own
// (threads below kP1 - kOwn): P1 index i1 and P2 index i2 of p1_point(kOwn + t).
struct HaloPoint {
    bool has;
    int i1, i2;
};
__device__ __forceinline__ HaloPoint halo_point()
{
    HaloPoint h{threadIdx.x < kP1 - kOwn, 0, 0};
    if (h.has) {
        int hx1, hy1;
        p1_point(kOwn + threadIdx.x, hx1, hy1);
        h.i1 = hx1 + kHX1 * hy1;
        h.i2 = (hx1 + 1) + kHX2 * (hy1 + 1);
    }
    return h;
}

// Predictor at one point of the plane whose input neighbourhood is (lo, mid,
// hi): n^P into pslot[i1], the rate into r.
template <typename Real>
__device__ __forceinline__ void predict_point(const FDPar<Real>& par, const Real* lo, const Real* mid, const Real* hi,
                                              int i1, int i2, Real* pslot, Real r[3], int side,
                                              const unsigned char* mmid = nullptr)
{
    Real nn[7][3], uu[7][3], np[3];
    if (mmid != nullptr && mmid[i2]) {  // obstacle: the director is held
        Real u0[3];
        split_pt(mid, i2, np, u0);
        r[0] = r[1] = r[2] = Real(0);
        st3(pslot, i1, np);
        return;
    }
    gather_slots(lo, mid, hi, i2, nn, uu);
    director_rate(nn, uu, par, r, (const Real*)nullptr, side);
#pragma unroll
    for (int a = 0; a < 3; ++a) np[a] = nn[0][a] + par.dt * r[a];
    if (par.renorm_p) {
        const Real inv = Real(1) / sqrt(np[0] * np[0] + np[1] * np[1] + np[2] * np[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) np[a] *= inv;
    }
    st3(pslot, i1, np);
}

// Kernel A, predictor on one plane: the thread's own point (rate kept in
// rown) and, with halo, its halo point.  The planes just below and above a
// chunk need n^P only at the tile's own points (halo = false).
template <typename Real>
__device__ __forceinline__ void predict_plane(const FDPar<Real>& par, const Real* lo, const Real* mid, const Real* hi,
                                              Real* pslot, int i1, int i2, const HaloPoint& hp, bool halo, Real rown[3],
                                              int side, const unsigned char* mmid = nullptr)
{
    predict_point(par, lo, mid, hi, i1, i2, pslot, rown, side, mmid);
    if (halo && hp.has) {
        Real r[3];
        predict_point(par, lo, mid, hi, hp.i1, hp.i2, pslot, r, side, mmid);
    }
}

// Ring slots: plane p of the input ring (6 kP2 Reals) and of the predictor
// ring (4 kP1 Reals) sits in slot slot3(p); the kernels rotate three slot
// indices (planes z - 1, z, z + 1) instead of recomputing them.
template <typename Real, bool Solid = false>
__device__ void fused_a_tile(const FDChan<Real>& c, const Real* __restrict__ nin, Real* __restrict__ nout, int tile)
{
    extern __shared__ __align__(16) unsigned char smem_fd[];
    Real* in = reinterpret_cast<Real*>(smem_fd);  // 3 slots x 6 x kP2 (input planes)
    Real* pr = in + 3 * 6 * kP2;                  // 3 slots x 4 x kP1 (predictor n^P)
    unsigned char* mk = reinterpret_cast<unsigned char*>(pr + 3 * 4 * kP1);  // 3 slots x kP2 obstacle masks
    const Geom& g = c.g;
    const int ntx = (g.nx + kTX - 1) / kTX, nty = (g.ny + kTY - 1) / kTY;
    const int tx_t = tile % ntx, ty_t = (tile / ntx) % nty, zc = tile / (ntx * nty);
    const int x0 = tx_t * kTX, y0 = ty_t * kTY;
    const int zch = fused_zchunk(c);
    const int zb = zc * zch, ze = min(zb + zch, g.nz);
    const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
    const bool active = threadIdx.x < kTX * kTY && x0 + tx < g.nx && y0 + ty < g.ny;
    const int N = g.N;
    const int i1 = (tx + 1) + kHX1 * (ty + 1);
    const int i2 = (tx + 2) + kHX2 * (ty + 2);
    const HaloPoint hp = halo_point();
    const PlaneMap pm = plane_map(g, x0, y0);
    const bool homeo = g.anchoring == NH_ANCHOR_HOMEOTROPIC;
    auto IN = [&](int sl) { return in + sl * (6 * kP2); };
    auto MK = [&](int sl) -> const unsigned char* { return Solid ? mk + sl * kP2 : nullptr; };
    unsigned char sv[kPts];
    auto PR = [&](int sl) { return pr + sl * (4 * kP1); };
    const int s0 = slot3(zb - 2), s1 = slot3(zb - 1), s2 = slot3(zb);
    Real v[kPts][6];
    prefetch_plane<Real, Solid>(nin, c.u, g, pm, zb - 2, v, c.solid, sv);
    commit_plane<Real, Solid>(pm, v, IN(s0), sv, mk + s0 * kP2);
    prefetch_plane<Real, Solid>(nin, c.u, g, pm, zb - 1, v, c.solid, sv);
    commit_plane<Real, Solid>(pm, v, IN(s1), sv, mk + s1 * kP2);
    prefetch_plane<Real, Solid>(nin, c.u, g, pm, zb, v, c.solid, sv);
    commit_plane<Real, Solid>(pm, v, IN(s2), sv, mk + s2 * kP2);
    prefetch_plane<Real, Solid>(nin, c.u, g, pm, zb + 1, v, c.solid, sv);  // in flight during the first predictor plane
    __syncthreads();
    Real rcur[3] = {0, 0, 0}, rnext[3] = {0, 0, 0};  // predictor rate at the own point, planes z and z + 1
    if (!is_ghost_plane(g, zb - 1))
        predict_plane(c.p, IN(s0), IN(s1), IN(s2), PR(s1), i1, i2, hp, false, rnext, free_plate_side(g, zb - 1),
                      MK(s1));
    // u one layer below the corrector's plane, at the thread's own point, carried in registers
    Real ulo[3], nc[3];
    split_pt(IN(s1), i2, nc, ulo);
    __syncthreads();  // plane zb - 2 is no longer read
    commit_plane<Real, Solid>(pm, v, IN(s0), sv, mk + s0 * kP2);  // plane zb + 1
    prefetch_plane<Real, Solid>(nin, c.u, g, pm, zb + 2, v, c.solid, sv);
    __syncthreads();
    if (!is_ghost_plane(g, zb))
        predict_plane(c.p, IN(s1), IN(s2), IN(s0), PR(s2), i1, i2, hp, true, rcur, free_plate_side(g, zb),
                      MK(s2));
    int sa = s1, sb = s2, sc = s0;  // slots of planes z - 1, z, z + 1 (plane z + 2 takes sa)
    for (int z = zb; z < ze; ++z) {
        __syncthreads();  // plane z - 1 is no longer read; its slot takes plane z + 2
        commit_plane<Real, Solid>(pm, v, IN(sa), sv, mk + sa * kP2);
        __syncthreads();
        if (z + 1 < ze) prefetch_plane<Real, Solid>(nin, c.u, g, pm, z + 3, v, c.solid, sv);  // overlaps the two evaluations below
        if (!is_ghost_plane(g, z + 1))
            predict_plane(c.p, IN(sb), IN(sc), IN(sa), PR(sc), i1, i2, hp, z + 1 < ze, rnext, free_plate_side(g, z + 1),
                          MK(sc));
        __syncthreads();
        if (active) {
            const Real* mid = PR(sb);
            // predictor of the planes above and below; at a plate the ghost
            // value (z_hat, or the adjacent fluid layer without anchoring)
            const bool glo = is_ghost_plane(g, z - 1), ghi = is_ghost_plane(g, z + 1);
            const Real* lo = glo ? mid : PR(sa);
            const Real* hi = ghi ? mid : PR(sc);
            const Real* inm = IN(sb);
            const Real* inh = IN(sc);
            Real nn[7][3], uu[7][3], r[3], n0[3], dummy[3];
            ld3(mid, i1, nn[0]);
            ld3(mid, i1 + 1, nn[1]);
            ld3(mid, i1 - 1, nn[2]);
            ld3(mid, i1 + kHX1, nn[3]);
            ld3(mid, i1 - kHX1, nn[4]);
            ld3(hi, i1, nn[5]);
            ld3(lo, i1, nn[6]);
            if (homeo) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (ghi) nn[5][a] = Real(a == 2 ? 1 : 0);
                    if (glo) nn[6][a] = Real(a == 2 ? 1 : 0);
                }
            }
            split_pt(inm, i2, n0, uu[0]);
            split_pt(inm, i2 + 1, dummy, uu[1]);
            split_pt(inm, i2 - 1, dummy, uu[2]);
            split_pt(inm, i2 + kHX2, dummy, uu[3]);
            split_pt(inm, i2 - kHX2, dummy, uu[4]);
            split_pt(inh, i2, dummy, uu[5]);
#pragma unroll
            for (int a = 0; a < 3; ++a) uu[6][a] = ulo[a];
            director_rate(nn, uu, c.p, r, (const Real*)nullptr, free_plate_side(g, z));
            Real nw[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) nw[a] = n0[a] + c.p.dt * Real(0.5) * (rcur[a] + r[a]);
            Real inv = Real(1) / sqrt(nw[0] * nw[0] + nw[1] * nw[1] + nw[2] * nw[2]);
            if (Solid && MK(sb)[i2]) {  // obstacle: the director is held
#pragma unroll
                for (int a = 0; a < 3; ++a) nw[a] = n0[a];
                inv = Real(1);
            }
            const int s = (x0 + tx) + g.nx * ((y0 + ty) + g.ny * z);
#pragma unroll
            for (int a = 0; a < 3; ++a) nout[a * N + s] = nw[a] * inv;
#pragma unroll
            for (int a = 0; a < 3; ++a) ulo[a] = uu[0][a];  // u of plane z: the next plane's lower neighbour
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) rcur[a] = rnext[a];
        const int t = sa;
        sa = sb;
        sb = sc;
        sc = t;
    }
}

// Kernel B tile: stress on plane p from planes p - 1, p, p + 1 of the 3-slot
// input ring.  The divergence at a tile point needs sigma_ax at its x
// neighbours and sigma_ay at its y neighbours in the same plane (into slot:
// sigma_.x then sigma_.y, 4 kP1 Reals each), and sigma_az of the point itself
// in the planes above and below, which stays in the registers of the thread
// that owns the point (szown).
template <typename Real>
__device__ __forceinline__ void stress_point_plane(const FDPar<Real>& par, const Real* lo, const Real* mid,
                                                   const Real* hi, int i1, int i2, Real* slot, Real sz[3], int side,
                                                   const unsigned char* mmid = nullptr)
{
    Real nn[7][3], uu[7][3], sig[9];
    if (mmid != nullptr && mmid[i2]) {  // obstacle: zero stress
#pragma unroll
        for (int k = 0; k < 9; ++k) sig[k] = Real(0);
    } else {
        gather_slots(lo, mid, hi, i2, nn, uu);
        stress_point(nn, uu, par, sig, (const Real*)nullptr, (const Real*)nullptr, side);
    }
    const Real sx[3] = {sig[0], sig[3], sig[6]}, sy[3] = {sig[1], sig[4], sig[7]};
    st3(slot, i1, sx);
    st3(slot + 4 * kP1, i1, sy);
    sz[0] = sig[2];
    sz[1] = sig[5];
    sz[2] = sig[8];
}

// Stress on one plane: zero sigma_az on a ghost plane; otherwise the own point
// and, with halo, the thread's halo point (the planes just below and above a
// chunk give only sigma_az: halo = false).
template <typename Real>
__device__ __forceinline__ void stress_plane(const FDChan<Real>& c, int p, const Real* lo, const Real* mid,
                                             const Real* hi, Real* slot, int i1, int i2, bool halo, Real szown[3],
                                             const unsigned char* mmid = nullptr)
{
    if (is_ghost_plane(c.g, p)) {
#pragma unroll
        for (int a = 0; a < 3; ++a) szown[a] = Real(0);
        return;
    }
    const int side = free_plate_side(c.g, p);
    stress_point_plane(c.p, lo, mid, hi, i1, i2, slot, szown, side, mmid);
    const HaloPoint hp = halo_point();  // recomputed here: kernel B runs at the register limit
    if (halo && hp.has) {
        Real sz[3];
        stress_point_plane(c.p, lo, mid, hi, hp.i1, hp.i2, slot, sz, side, mmid);
    }
}

// Diag: the kernel also leaves the diagnostics' block partials of the updated
// director it holds (BDiag): per own site the lattice link energy to its x+1,
// y+1 and z+1 neighbours (and from the lower ghost layer at a homeotropic
// plate), the site terms, |n| and the tube weight (1 - n_z)/2, as the
// director-only diagnostics kernels sum them.
template <typename Real, bool Solid = false, bool Diag = false>
__device__ void fused_b_tile(const FDChan<Real>& c, const Real* __restrict__ nin, Real* __restrict__ ncopy, int tile,
                             const BDiag* bd = nullptr)
{
    extern __shared__ __align__(16) unsigned char smem_fd[];
    Real* in = reinterpret_cast<Real*>(smem_fd);  // 3 slots x 6 x kP2 (input planes)
    Real* sg = in + 3 * 6 * kP2;                  // 2 slots x 8 x kP1 (sigma_.x, sigma_.y), slot z & 1
    unsigned char* mk = reinterpret_cast<unsigned char*>(sg + 2 * 8 * kP1);  // 3 slots x kP2 obstacle masks
    const Geom& g = c.g;
    const int ntx = (g.nx + kTX - 1) / kTX, nty = (g.ny + kTY - 1) / kTY;
    const int tx_t = tile % ntx, ty_t = (tile / ntx) % nty, zc = tile / (ntx * nty);
    const int x0 = tx_t * kTX, y0 = ty_t * kTY;
    const int zch = fused_zchunk(c);
    const int zb = zc * zch, ze = min(zb + zch, g.nz);
    const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
    const bool active = threadIdx.x < kTX * kTY && x0 + tx < g.nx && y0 + ty < g.ny;
    const int N = g.N;
    const int i1 = (tx + 1) + kHX1 * (ty + 1);
    const int i2 = (tx + 2) + kHX2 * (ty + 2);
    const PlaneMap pm = plane_map(g, x0, y0);
    auto IN = [&](int sl) { return in + sl * (6 * kP2); };
    auto MK = [&](int sl) -> const unsigned char* { return Solid ? mk + sl * kP2 : nullptr; };
    unsigned char sv[kPts];
    auto SG = [&](int p) { return sg + (p & 1) * (8 * kP1); };
    const int s0 = slot3(zb - 2), s1 = slot3(zb - 1), s2 = slot3(zb);
    Real v[kPts][6];
    prefetch_plane<Real, Solid>(nin, c.u, g, pm, zb - 2, v, c.solid, sv);
    commit_plane<Real, Solid>(pm, v, IN(s0), sv, mk + s0 * kP2);
    prefetch_plane<Real, Solid>(nin, c.u, g, pm, zb - 1, v, c.solid, sv);
    commit_plane<Real, Solid>(pm, v, IN(s1), sv, mk + s1 * kP2);
    prefetch_plane<Real, Solid>(nin, c.u, g, pm, zb, v, c.solid, sv);
    commit_plane<Real, Solid>(pm, v, IN(s2), sv, mk + s2 * kP2);
    prefetch_plane<Real, Solid>(nin, c.u, g, pm, zb + 1, v, c.solid, sv);  // in flight during the first stress plane
    __syncthreads();
    Real szlo[3], szmid[3], szhi[3];  // sigma_az at the own point, planes z - 1, z, z + 1
    stress_plane(c, zb - 1, IN(s0), IN(s1), IN(s2), SG(zb - 1), i1, i2, false, szlo, MK(s1));
    __syncthreads();  // plane zb - 2 is no longer read
    commit_plane<Real, Solid>(pm, v, IN(s0), sv, mk + s0 * kP2);  // plane zb + 1
    prefetch_plane<Real, Solid>(nin, c.u, g, pm, zb + 2, v, c.solid, sv);
    __syncthreads();
    stress_plane(c, zb, IN(s1), IN(s2), IN(s0), SG(zb), i1, i2, true, szmid, MK(s2));
    int sa = s1, sb = s2, sc = s0;  // input slots of planes z - 1, z, z + 1 (plane z + 2 takes sa)
    Real d_e = 0, d_w = 0, d_mn = Real(1e30), d_mx = 0;  // Diag: energy, tube weight, |n| extrema of the column
    int d_bad = 0;
    for (int z = zb; z < ze; ++z) {
        __syncthreads();  // plane z - 1 is no longer read; its slots take planes z + 2 (input), z + 1 (sigma)
        commit_plane<Real, Solid>(pm, v, IN(sa), sv, mk + sa * kP2);
        __syncthreads();
        if (z + 1 < ze) prefetch_plane<Real, Solid>(nin, c.u, g, pm, z + 3, v, c.solid, sv);
        stress_plane(c, z + 1, IN(sb), IN(sc), IN(sa), SG(z + 1), i1, i2, z + 1 < ze, szhi, MK(sc));
        __syncthreads();
        if (active) {
            const Real* sx = SG(z);
            const Real* sy = sx + 4 * kP1;
            Real xp[3], xm[3], yp[3], ym[3];
            ld3(sx, i1 + 1, xp);
            ld3(sx, i1 - 1, xm);
            ld3(sy, i1 + kHX1, yp);
            ld3(sy, i1 - kHX1, ym);
            const int s = (x0 + tx) + g.nx * ((y0 + ty) + g.ny * z);
            // ghost planes hold zero sigma_az; mirror: the wall layer's own
            const bool mlo = c.p.mirror && is_ghost_plane(g, z - 1), mhi = c.p.mirror && is_ghost_plane(g, z + 1);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const Real hi = mhi ? szmid[a] : szhi[a], lo = mlo ? szmid[a] : szlo[a];
                c.F[a * N + s] = (Solid && MK(sb)[i2]) ? Real(0)  // no force on an obstacle node
                                                        : Real(0.5) * ((xp[a] - xm[a]) + (yp[a] - ym[a]) + (hi - lo));
            }
            if (ncopy || Diag) {
                Real n0[3], u0[3];
                split_pt(IN(sb), i2, n0, u0);
                if (ncopy) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) ncopy[a * N + s] = n0[a];
                }
                if constexpr (Diag) {
                    const Real K = c.p.K, q0 = c.p.q0;
                    Real nx[3], ny[3], nz[3];
                    ld_n(IN(sb), i2 + 1, nx);
                    ld_n(IN(sb), i2 + kHX2, ny);
                    ld_n(IN(sc), i2, nz);  // plane z + 1 (the ghost layer above the top plate)
                    Real e = dsum::link_energy(n0, nx, 0, K, q0);
                    e += dsum::link_energy(n0, ny, 1, K, q0);
                    e += dsum::link_energy(n0, nz, 2, K, q0);
                    if (g.walls && z == 0 && g.anchoring == NH_ANCHOR_HOMEOTROPIC) {
                        const Real zh[3] = {Real(0), Real(0), Real(1)};  // the ghost layer below
                        e += dsum::link_energy(zh, n0, 2, K, q0);
                    }
                    d_e += e + (Real(0.5) * K * q0 * q0 - Real(0.5) * c.p.W0 * (n0[2] * n0[2]));
                    const Real nm = dsum::norm3(n0);
                    d_mn = min(d_mn, nm);
                    d_mx = max(d_mx, nm);
                    d_bad += !isfinite(nm) ? 1 : 0;
                    d_w += Real(0.5) * (Real(1) - n0[2]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            szlo[a] = szmid[a];
            szmid[a] = szhi[a];
        }
        const int t = sa;
        sa = sb;
        sb = sc;
        sc = t;
    }
    if constexpr (Diag) {
        // the planes are no longer read: the per-warp tube sums and the
        // previous centroids take the start of the dynamic shared memory
        const int T = bd->n_tubes;
        __syncthreads();
        Real(*tube_acc)[NH_MAX_TUBES * 5] = reinterpret_cast<Real(*)[NH_MAX_TUBES * 5]>(smem_fd);
        float(*txy)[2] = reinterpret_cast<float(*)[2]>(smem_fd + sizeof(Real) * (kFusedThreads / 32) * NH_MAX_TUBES * 5);
        for (int k = threadIdx.x; k < (kFusedThreads / 32) * NH_MAX_TUBES * 5; k += blockDim.x) (&tube_acc[0][0])[k] = Real(0);
        for (int k = threadIdx.x; k < T; k += blockDim.x) {
            txy[k][0] = (float)bd->tubes[2 * k];
            txy[k][1] = (float)bd->tubes[2 * k + 1];
        }
        __syncthreads();
        if (T > 0) {
            int owner = -1;
            Real v[5] = {0, 0, 0, 0, 0};
            if (active) {
                owner = dsum::nearest_tube(g, bd->tubes, txy, T, x0 + tx, y0 + ty);
                dsum::tube_values(g, bd->trig, x0 + tx, y0 + ty, d_w, v);
            }
            dsum::warp_tube_accumulate(owner, v, threadIdx.x & 31, tube_acc[threadIdx.x >> 5]);
        }
        dsum::block_partials<kFusedThreads>(bd->partials, bd->lbpart, bd->lbp_blocks, Real(0), d_e, Real(0), d_mn,
                                            d_mx, d_bad, tube_acc, T);
    }
}

// Solid: the channel has obstacles (held directors, no-slip, zero stress and
// force at solid nodes, as the per-site kernels).
template <typename Real, bool Solid>
__global__ void __launch_bounds__(kFusedThreads, sizeof(Real) == 4 ? 4 : 2) fused_a_kernel(const FDChan<Real> c, const Real* nin, Real* nout)
{
    fused_a_tile<Real, Solid>(c, nin, nout, blockIdx.x);
}

// Fused B at three blocks per SM (up to 85 registers): 101 us against 116 us
// at four blocks of 64 registers on the 256x256x64 channel, FP32.
template <typename Real, bool Solid>
__global__ void __launch_bounds__(kFusedThreads, sizeof(Real) == 4 ? 3 : 2) fused_b_kernel(const FDChan<Real> c, const Real* nin, Real* ncopy)
{
    fused_b_tile<Real, Solid>(c, nin, ncopy, blockIdx.x);
}
// The same with the diagnostics partials of the updated director (no obstacles).
// Three blocks per SM, as fused B (measured on the 256x256x64 channel: 122 us
// against 137 us at four blocks of 64 registers).
template <typename Real>
__global__ void __launch_bounds__(kFusedThreads, sizeof(Real) == 4 ? 3 : 2)
    fused_b_diag_kernel(const FDChan<Real> c, const Real* nin, Real* ncopy, const BDiag bd)
{
    fused_b_tile<Real, false, true>(c, nin, ncopy, blockIdx.x, &bd);
}

// Batched fused kernels: a persistent grid walks the (channel, tile) work
// list; stage 0 = kernel A (n -> nP), 1 = kernel B (nP -> F, copy into n),
// 2 = kernel A (nP -> n), for relaxations that alternate the two buffers.
template <typename Real, int Stage, bool Solid>
__global__ void __launch_bounds__(kFusedThreads, sizeof(Real) == 4 ? 3 : 2) fused_batch_kernel(const FDBatch<Real> b)
{
    const int total = b.prefix[b.count];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int lo = 0, hi = b.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.prefix[mid] <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        const FDChan<Real>& c = b.ch[lo];
        if (Stage == 0)
            fused_a_tile<Real, Solid>(c, c.n, c.nP, t - b.prefix[lo]);
        else if (Stage == 1)
            fused_b_tile<Real, Solid>(c, c.nP, c.n, t - b.prefix[lo]);
        else
            fused_a_tile<Real, Solid>(c, c.nP, c.n, t - b.prefix[lo]);
        __syncthreads();
    }
}

template <typename Real>
inline int fused_tiles(const FDChan<Real>& c)
{
    const int zch = fused_zchunk(c);
    return fused_xy_tiles(c.g) * ((c.g.nz + zch - 1) / zch);
}

template <typename Real>
cudaError_t prepare_fused()
{
    static bool done = false;  // the attribute is per function; setting it twice is harmless
    if (done) return cudaSuccess;
    const int a = (int)fused_a_smem<Real>(), b = (int)fused_b_smem<Real>();
    const cudaFuncAttribute attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(fused_a_kernel<Real, false>, attr, a);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fused_a_kernel<Real, true>, attr, a);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fused_b_kernel<Real, false>, attr, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fused_b_kernel<Real, true>, attr, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fused_b_diag_kernel<Real>, attr, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fused_batch_kernel<Real, 0, false>, attr, a);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fused_batch_kernel<Real, 0, true>, attr, a);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fused_batch_kernel<Real, 1, false>, attr, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fused_batch_kernel<Real, 1, true>, attr, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fused_batch_kernel<Real, 2, false>, attr, a);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fused_batch_kernel<Real, 2, true>, attr, a);
    if (e == cudaSuccess) done = true;
    return e;
}

inline int blocks_for(int N) { return (N + 255) / 256; }

}  // namespace

template <typename Real>
cudaError_t launch_fd_batch(FDBatch<Real>& b, int stage, int grid, cudaStream_t st)
{
    if (b.count < 1 || b.count > kMaxBatch) return cudaErrorInvalidValue;
    b.prefix[0] = 0;
    for (int k = 0; k < b.count; ++k) b.prefix[k + 1] = b.prefix[k] + blocks_for(b.ch[k].g.N);
    const int blocks = grid < b.prefix[b.count] ? grid : b.prefix[b.count];
    switch (stage) {
    case 0: fd_batch_kernel<Real, 0><<<blocks, 256, 0, st>>>(b); break;
    case 1: fd_batch_kernel<Real, 1><<<blocks, 256, 0, st>>>(b); break;
    case 2: fd_batch_kernel<Real, 2><<<blocks, 256, 0, st>>>(b); break;
    case 3: fd_batch_kernel<Real, 3><<<blocks, 256, 0, st>>>(b); break;
    case 4: fd_batch_kernel<Real, 4><<<blocks, 256, 0, st>>>(b); break;  // three-constant P stage from n
    case 5: fd_batch_kernel<Real, 5><<<blocks, 256, 0, st>>>(b); break;  // ... and from n^P
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
template cudaError_t launch_fd_batch<double>(FDBatch<double>&, int, int, cudaStream_t);
template cudaError_t launch_fd_batch<float>(FDBatch<float>&, int, int, cudaStream_t);

template <typename Real>
cudaError_t launch_fd_predict(const FDChan<Real>& c, cudaStream_t st)
{
    fd_kernel<Real, 0><<<blocks_for(c.g.N), 256, 0, st>>>(c);
    return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_fd_correct(const FDChan<Real>& c, cudaStream_t st)
{
    fd_kernel<Real, 1><<<blocks_for(c.g.N), 256, 0, st>>>(c);
    return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_stress(const FDChan<Real>& c, cudaStream_t st)
{
    fd_kernel<Real, 2><<<blocks_for(c.g.N), 256, 0, st>>>(c);
    return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_force(const FDChan<Real>& c, cudaStream_t st)
{
    fd_kernel<Real, 3><<<blocks_for(c.g.N), 256, 0, st>>>(c);
    return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_frank3_p(const FDChan<Real>& c, bool from_predictor, cudaStream_t st)
{
    if (c.P3 == nullptr) return cudaErrorInvalidValue;
    if (from_predictor)
        fd_kernel<Real, 5><<<blocks_for(c.g.N), 256, 0, st>>>(c);
    else
        fd_kernel<Real, 4><<<blocks_for(c.g.N), 256, 0, st>>>(c);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_fd_fused_a(const FDChan<Real>& c, const Real* nin, Real* nout, cudaStream_t st)
{
    cudaError_t e = prepare_fused<Real>();
    if (e != cudaSuccess) return e;
    if (c.solid != nullptr)
        fused_a_kernel<Real, true><<<fused_tiles(c), kFusedThreads, fused_a_smem<Real>(), st>>>(c, nin, nout);
    else
        fused_a_kernel<Real, false><<<fused_tiles(c), kFusedThreads, fused_a_smem<Real>(), st>>>(c, nin, nout);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_fd_fused_b(const FDChan<Real>& c, const Real* nin, Real* ncopy, cudaStream_t st, const BDiag* diag)
{
    cudaError_t e = prepare_fused<Real>();
    if (e != cudaSuccess) return e;
    if (diag != nullptr) {
        if (c.solid != nullptr || diag->n_tubes < 0 || diag->n_tubes > NH_MAX_TUBES) return cudaErrorInvalidValue;
        fused_b_diag_kernel<Real><<<fused_tiles(c), kFusedThreads, fused_b_smem<Real>(), st>>>(c, nin, ncopy, *diag);
    } else if (c.solid != nullptr) {
        fused_b_kernel<Real, true><<<fused_tiles(c), kFusedThreads, fused_b_smem<Real>(), st>>>(c, nin, ncopy);
    } else {
        fused_b_kernel<Real, false><<<fused_tiles(c), kFusedThreads, fused_b_smem<Real>(), st>>>(c, nin, ncopy);
    }
    return cudaGetLastError();
}

template <typename Real>
int fd_fused_tiles(const FDChan<Real>& c)
{
    return fused_tiles(c);
}

template <typename Real>
cudaError_t launch_fd_fused_batch(FDBatch<Real>& b, int stage, int grid, cudaStream_t st)
{
    if (b.count < 1 || b.count > kMaxBatch) return cudaErrorInvalidValue;
    cudaError_t e = prepare_fused<Real>();
    if (e != cudaSuccess) return e;
    long long tile_layers = 0;
    for (int k = 0; k < b.count; ++k) tile_layers += (long long)b.ch[k].g.nz * fused_xy_tiles(b.ch[k].g);
    const int zch = zchunk_for(tile_layers);
    b.prefix[0] = 0;
    for (int k = 0; k < b.count; ++k) {
        b.ch[k].zch = zch;
        b.prefix[k + 1] = b.prefix[k] + fused_tiles(b.ch[k]);
    }
    const int blocks = grid < b.prefix[b.count] ? grid : b.prefix[b.count];
    const size_t smem = stage == 1 ? fused_b_smem<Real>() : fused_a_smem<Real>();
    bool solid = false;
    for (int k = 0; k < b.count; ++k) solid = solid || b.ch[k].solid != nullptr;
    if (solid) {
        switch (stage) {
        case 0: fused_batch_kernel<Real, 0, true><<<blocks, kFusedThreads, smem, st>>>(b); break;
        case 1: fused_batch_kernel<Real, 1, true><<<blocks, kFusedThreads, smem, st>>>(b); break;
        default: fused_batch_kernel<Real, 2, true><<<blocks, kFusedThreads, smem, st>>>(b); break;
        }
    } else {
        switch (stage) {
        case 0: fused_batch_kernel<Real, 0, false><<<blocks, kFusedThreads, smem, st>>>(b); break;
        case 1: fused_batch_kernel<Real, 1, false><<<blocks, kFusedThreads, smem, st>>>(b); break;
        default: fused_batch_kernel<Real, 2, false><<<blocks, kFusedThreads, smem, st>>>(b); break;
        }
    }
    return cudaGetLastError();
}

template cudaError_t launch_fd_fused_a<double>(const FDChan<double>&, const double*, double*, cudaStream_t);
template cudaError_t launch_fd_fused_a<float>(const FDChan<float>&, const float*, float*, cudaStream_t);
template cudaError_t launch_fd_fused_b<double>(const FDChan<double>&, const double*, double*, cudaStream_t,
                                                const BDiag*);
template int fd_fused_tiles<double>(const FDChan<double>&);
template cudaError_t launch_fd_fused_b<float>(const FDChan<float>&, const float*, float*, cudaStream_t, const BDiag*);
template int fd_fused_tiles<float>(const FDChan<float>&);
template cudaError_t launch_fd_fused_batch<double>(FDBatch<double>&, int, int, cudaStream_t);
template cudaError_t launch_fd_fused_batch<float>(FDBatch<float>&, int, int, cudaStream_t);

template cudaError_t launch_fd_predict<double>(const FDChan<double>&, cudaStream_t);
template cudaError_t launch_fd_predict<float>(const FDChan<float>&, cudaStream_t);
template cudaError_t launch_fd_correct<double>(const FDChan<double>&, cudaStream_t);
template cudaError_t launch_fd_correct<float>(const FDChan<float>&, cudaStream_t);
template cudaError_t launch_stress<double>(const FDChan<double>&, cudaStream_t);
template cudaError_t launch_stress<float>(const FDChan<float>&, cudaStream_t);
template cudaError_t launch_force<double>(const FDChan<double>&, cudaStream_t);
template cudaError_t launch_force<float>(const FDChan<float>&, cudaStream_t);
template cudaError_t launch_frank3_p<double>(const FDChan<double>&, bool, cudaStream_t);
template cudaError_t launch_frank3_p<float>(const FDChan<float>&, bool, cudaStream_t);

}  // namespace nh
