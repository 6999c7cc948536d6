/*
 * FP64 CPU oracle of the interpolation-based discrete imaging model H = D G and of its
 * adjoint H^T = G^T D^T (Sec. II.B and the Appendix of Wang et al., "Accelerating image
 * reconstruction in three-dimensional optoacoustic tomography on graphics processing units").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, __graft_entry__.smoke() and the cpu_baseline leg
 * of bench.py load this library.  It shares no code with the CUDA path: it is written straight
 * from the paper's definitions, plain and slow, in double precision, with no blocking or
 * reordering beyond what the definitions state.  The only pruning (oracle_Gt_nodes) skips
 * terms that are provably zero by the triangle inequality and is itself checked against the
 * full scatter in the tests.
 *
 * Conventions (shared with the inputs, not with the GPU code):
 *   volume alpha[(iz*ny + iy)*nx + ix], node n at r_n = origin + ds*(ix, iy, iz)   (Eq. coeffint)
 *   data   g[q*K + k], t_k = t_min + k*dt, dt = 1/fs                              (Eq. CDmodel)
 *   rho_k = c*t_k is the radius of the shell of sample k                          (Eq. srt)
 *
 * Readings of the paper taken here (where it is silent or inconsistent):
 *   - lattice: theta_i = i*dtheta, i < N_i = floor(theta_max/dtheta); phi_j = j*dphi_i,
 *     j < N_j = floor(2 pi/dphi_i); dtheta = ds/rho, dphi_i = ds/(rho sin theta_i)  (Appendix)
 *   - local frame of transducer q: e_z = -r_q/|r_q| (towards the origin), e_y = unit(z x r_q)
 *     ((0,1,0) if r_q is on the z axis), e_x = e_y x e_z                         (Appendix)
 *   - theta_max = acos((|r_q|^2 + rho^2 - R^2)/(2 rho |r_q|)); argument > 1: no points;
 *     argument < -1: theta_max = pi; rho <= 0: no points                          (Alg. 4 / Appendix)
 *   - the expansion function is zero outside its support, nodes outside the grid do not
 *     exist, so the interpolant is exactly sum_n alpha_n psi_n(r)                 (Eq. expfunI)
 *   - D uses tau_k = t_min/dt + k; rows 0 and K-1 are zero; a term with tau <= 0 is zero
 *                                                                                 (Eq. dis_g2p)
 *   - D^T is the exact transpose of that D (masked neighbours), not the paper's printed loop.
 *   - point weights (Eq. dis_srt): ds^2 for every point (area = 0), or, with area = 1, the
 *     area of ring i's strip of the shell shared by its points, ds * 2 pi rho sin(theta_i) / N_j
 *     (the strip has polar width dtheta, i.e. ds on the shell, and circumference
 *     2 pi rho sin(theta_i)); the latter removes the bias of rounding 2 pi / dphi_i down to N_j.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;
    double ds;          /* grid spacing Delta_s (mm) */
    double origin[3];   /* position of node (0,0,0) (mm) */
    int nq;             /* number of transducers Q */
    const double *pos;  /* [Q][3] transducer positions (mm) */
    int nk;             /* samples per transducer K */
    double fs;          /* sampling rate (MHz) */
    double tmin;        /* time of sample 0 (us) */
    double c;           /* speed of sound (mm/us) */
    double R;           /* support radius (mm) */
    double gamma;       /* Grueneisen coefficient Gamma = beta c^2 / C_p */
    int area;           /* 0: weight ds^2 per lattice point; 1: exact strip area per point */
} orc_geom;

/* ------------------------------------------------------------------ geometry (Appendix) */

/* Local frame of a transducer: z axis towards the global origin. */
static void transducer_frame(const double r[3], double ex[3], double ey[3], double ez[3], double *rs)
{
    double n = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    *rs = n;
    ez[0] = -r[0] / n; ez[1] = -r[1] / n; ez[2] = -r[2] / n;
    /* z-hat x r-hat = (-r_y, r_x, 0)/|r| */
    double a = -r[1] / n, b = r[0] / n;
    double m = sqrt(a * a + b * b);
    if (m > 0.0) { ey[0] = a / m; ey[1] = b / m; ey[2] = 0.0; }
    else { ey[0] = 0.0; ey[1] = 1.0; ey[2] = 0.0; }
    ex[0] = ey[1] * ez[2] - ey[2] * ez[1];
    ex[1] = ey[2] * ez[0] - ey[0] * ez[2];
    ex[2] = ey[0] * ez[1] - ey[1] * ez[0];
}

/* Shell of sample k for a transducer at distance rs from the origin: returns the number of
 * rings N_i (0 if the shell misses the support sphere) and the shell radius and dtheta. */
static int shell_rings(const orc_geom *g, double rs, int k, double *rho_out, double *dth_out)
{
    double dt = 1.0 / g->fs;
    double t = g->tmin + k * dt;
    double rho = g->c * t;
    *rho_out = rho; *dth_out = 0.0;
    if (!(rho > 0.0)) return 0;
    double arg = (rs * rs + rho * rho - g->R * g->R) / (2.0 * rho * rs);
    if (arg > 1.0) return 0;
    double thmax = (arg < -1.0) ? M_PI : acos(arg);
    double dth = g->ds / rho;
    *dth_out = dth;
    return (int)floor(thmax / dth);
}

/* Number of azimuthal points N_j on ring i and the azimuthal step dphi_i. */
static int ring_points(const orc_geom *g, double rho, double th, double *dph_out)
{
    double st = sin(th);
    double dph = g->ds / (rho * st);   /* +inf at the pole: no points */
    *dph_out = dph;
    return (int)floor(2.0 * M_PI / dph);
}

/* Weight of each point of ring i relative to ds^2: 1, or with exact strip areas
 * (ds * 2 pi rho sin(theta_i) / N_j) / ds^2. */
static double ring_weight(const orc_geom *g, double rho, double th, int nj)
{
    if (!g->area || nj <= 0) return 1.0;
    return 2.0 * M_PI * rho * sin(th) / (nj * g->ds);
}

/* Global position (mm) of lattice point (k, i, j) of transducer q  (r_{k,i,j}, Appendix). */
static void lattice_point(const double rq[3], const double ex[3], const double ey[3], const double ez[3],
                          double rho, double th, double ph, double P[3])
{
    double st = sin(th), ct = cos(th), sp = sin(ph), cp = cos(ph);
    for (int d = 0; d < 3; ++d)
        P[d] = rq[d] + rho * (st * cp * ex[d] + st * sp * ey[d] + ct * ez[d]);
}

/* ------------------------------------------------------------------ interpolation (Eq. expfunI) */

/* f(P) = sum_n alpha_n psi_n(P) with the trilinear tent; only the 8 nodes around P can be
 * non-zero, nodes outside the grid are absent. */
static double interp(const orc_geom *g, const double *alpha, const double P[3])
{
    double x = (P[0] - g->origin[0]) / g->ds;
    double y = (P[1] - g->origin[1]) / g->ds;
    double z = (P[2] - g->origin[2]) / g->ds;
    double fx = floor(x), fy = floor(y), fz = floor(z);
    long ix = (long)fx, iy = (long)fy, iz = (long)fz;
    double wx = x - fx, wy = y - fy, wz = z - fz;
    double s = 0.0;
    for (int dz = 0; dz < 2; ++dz) {
        long jz = iz + dz;
        if (jz < 0 || jz >= g->nz) continue;
        double vz = dz ? wz : 1.0 - wz;
        for (int dy = 0; dy < 2; ++dy) {
            long jy = iy + dy;
            if (jy < 0 || jy >= g->ny) continue;
            double vy = dy ? wy : 1.0 - wy;
            for (int dx = 0; dx < 2; ++dx) {
                long jx = ix + dx;
                if (jx < 0 || jx >= g->nx) continue;
                double vx = dx ? wx : 1.0 - wx;
                s += alpha[(jz * g->ny + jy) * g->nx + jx] * vx * vy * vz;
            }
        }
    }
    return s;
}

/* Transpose of interp: add v * psi_n(P) to the 8 nodes around P. */
static void splat(const orc_geom *g, double *out, const double P[3], double v)
{
    double x = (P[0] - g->origin[0]) / g->ds;
    double y = (P[1] - g->origin[1]) / g->ds;
    double z = (P[2] - g->origin[2]) / g->ds;
    double fx = floor(x), fy = floor(y), fz = floor(z);
    long ix = (long)fx, iy = (long)fy, iz = (long)fz;
    double wx = x - fx, wy = y - fy, wz = z - fz;
    for (int dz = 0; dz < 2; ++dz) {
        long jz = iz + dz;
        if (jz < 0 || jz >= g->nz) continue;
        double vz = dz ? wz : 1.0 - wz;
        for (int dy = 0; dy < 2; ++dy) {
            long jy = iy + dy;
            if (jy < 0 || jy >= g->ny) continue;
            double vy = dy ? wy : 1.0 - wy;
            for (int dx = 0; dx < 2; ++dx) {
                long jx = ix + dx;
                if (jx < 0 || jx >= g->nx) continue;
                double vx = dx ? wx : 1.0 - wx;
                out[(jz * g->ny + jy) * g->nx + jx] += v * vx * vy * vz;
            }
        }
    }
}

/* ------------------------------------------------------------------ G (Eq. dis_srt) */

/* One data sample: g_{qK+k} = ds^2 * sum_{i<N_i} w_i sum_{j<N_j} f(r_{k,i,j}) (w_i = 1 unless
 * exact strip areas are asked for). */
static double G_sample(const orc_geom *g, const double *alpha, int q, int k)
{
    double ex[3], ey[3], ez[3], rs, rho, dth, dph;
    const double *rq = g->pos + 3 * q;
    transducer_frame(rq, ex, ey, ez, &rs);
    int ni = shell_rings(g, rs, k, &rho, &dth);
    double s = 0.0;
    for (int i = 0; i < ni; ++i) {
        double th = i * dth;
        int nj = ring_points(g, rho, th, &dph);
        double wi = ring_weight(g, rho, th, nj), si = 0.0;
        for (int j = 0; j < nj; ++j) {
            double P[3];
            lattice_point(rq, ex, ey, ez, rho, th, j * dph, P);
            si += interp(g, alpha, P);
        }
        s += wi * si;
    }
    return g->ds * g->ds * s;
}

void oracle_G(const orc_geom *g, const double *alpha, double *out)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < g->nq; ++q)
        for (int k = 0; k < g->nk; ++k)
            out[(long)q * g->nk + k] = G_sample(g, alpha, q, k);
}

/* Selected rows (q, k) of G alpha: rows[2*r], rows[2*r+1]. */
void oracle_G_rows(const orc_geom *g, const double *alpha, const int *rows, int nrows, double *out)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < nrows; ++r)
        out[r] = G_sample(g, alpha, rows[2 * r], rows[2 * r + 1]);
}

/* ------------------------------------------------------------------ G^T (adjoint of Eq. dis_srt) */

/* alpha'_n = ds^2 sum_q sum_k g'_{qK+k} sum_{i,j} psi_n(r_{k,i,j}) as the literal scatter. */
static void Gt_transducer(const orc_geom *g, const double *gp, int q, double *out)
{
    double ex[3], ey[3], ez[3], rs, rho, dth, dph;
    const double *rq = g->pos + 3 * q;
    transducer_frame(rq, ex, ey, ez, &rs);
    for (int k = 0; k < g->nk; ++k) {
        double v = g->ds * g->ds * gp[(long)q * g->nk + k];
        if (v == 0.0) continue;
        int ni = shell_rings(g, rs, k, &rho, &dth);
        for (int i = 0; i < ni; ++i) {
            double th = i * dth;
            int nj = ring_points(g, rho, th, &dph);
            double vi = v * ring_weight(g, rho, th, nj);
            for (int j = 0; j < nj; ++j) {
                double P[3];
                lattice_point(rq, ex, ey, ez, rho, th, j * dph, P);
                splat(g, out, P, vi);
            }
        }
    }
}

void oracle_Gt(const orc_geom *g, const double *gp, double *out)
{
    long N = (long)g->nx * g->ny * g->nz;
    memset(out, 0, sizeof(double) * N);
#ifdef _OPENMP
    int nt = omp_get_max_threads();
    if (nt > g->nq) nt = g->nq;
    if (nt > 1) {
        double *priv = (double *)calloc((size_t)nt * N, sizeof(double));
        if (priv) {
            #pragma omp parallel num_threads(nt)
            {
                double *mine = priv + (long)omp_get_thread_num() * N;
                #pragma omp for schedule(dynamic, 1)
                for (int q = 0; q < g->nq; ++q) Gt_transducer(g, gp, q, mine);
            }
            for (int t = 0; t < nt; ++t)
                for (long n = 0; n < N; ++n) out[n] += priv[(long)t * N + n];
            free(priv);
            return;
        }
    }
#endif
    for (int q = 0; q < g->nq; ++q) Gt_transducer(g, gp, q, out);
}

/* alpha'_n of G^T at selected nodes only.  Exact: a point P can have psi_n(P) > 0 only if
 * |P - r_n| < sqrt(3) ds, so (triangle inequality on the shell) only shells with
 * |rho - |r_n - r_q|| < sqrt(3) ds and, on a shell, only rings whose polar angle is within the
 * angle subtended by that ball can contribute; every point of those rings is evaluated. */
void oracle_Gt_nodes(const orc_geom *g, const double *gp, const int *nodes, int nn, double *out)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int m = 0; m < nn; ++m) {
        int ix = nodes[3 * m], iy = nodes[3 * m + 1], iz = nodes[3 * m + 2];
        double rn[3] = {g->origin[0] + g->ds * ix, g->origin[1] + g->ds * iy, g->origin[2] + g->ds * iz};
        double rad = sqrt(3.0) * g->ds;
        double s = 0.0;
        for (int q = 0; q < g->nq; ++q) {
            double ex[3], ey[3], ez[3], rs, rho, dth, dph;
            const double *rq = g->pos + 3 * q;
            transducer_frame(rq, ex, ey, ez, &rs);
            double v[3] = {rn[0] - rq[0], rn[1] - rq[1], rn[2] - rq[2]};
            double d = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            double thn = acos(fmax(-1.0, fmin(1.0, (v[0] * ez[0] + v[1] * ez[1] + v[2] * ez[2]) / d)));
            for (int k = 0; k < g->nk; ++k) {
                double w = gp[(long)q * g->nk + k];
                if (w == 0.0) continue;
                int ni = shell_rings(g, rs, k, &rho, &dth);
                if (ni == 0 || fabs(rho - d) >= rad) continue;
                /* angle between P - r_q and r_n - r_q must satisfy
                   rho^2 + d^2 - 2 rho d cos(angle) < rad^2 */
                double cmin = (rho * rho + d * d - rad * rad) / (2.0 * rho * d);
                double amax = cmin <= -1.0 ? M_PI : acos(fmin(1.0, cmin));
                double ss = 0.0;
                for (int i = 0; i < ni; ++i) {
                    double th = i * dth;
                    if (fabs(th - thn) > amax + 1e-9) continue;
                    int nj = ring_points(g, rho, th, &dph);
                    double si = 0.0;
                    for (int j = 0; j < nj; ++j) {
                        double P[3];
                        lattice_point(rq, ex, ey, ez, rho, th, j * dph, P);
                        double t = 1.0;
                        for (int dd = 0; dd < 3; ++dd) {
                            double u = fabs(P[dd] - rn[dd]) / g->ds;
                            t *= (u < 1.0) ? 1.0 - u : 0.0;
                        }
                        si += t;
                    }
                    ss += ring_weight(g, rho, th, nj) * si;
                }
                s += w * ss;
            }
        }
        out[m] = g->ds * g->ds * s;
    }
}

/* ------------------------------------------------------------------ D and D^T (Eq. dis_g2p) */

static double tau(const orc_geom *g, int k) { return g->tmin * g->fs + k; }   /* t_k / dt */

/* p_k = beta/(8 pi C_p dt^2) (g_{k+1}/tau_{k+1} - g_{k-1}/tau_{k-1}), beta/C_p = Gamma/c^2. */
void oracle_D(const orc_geom *g, const double *gin, double *out)
{
    double dt = 1.0 / g->fs;
    double cd = g->gamma / (8.0 * M_PI * g->c * g->c * dt * dt);
    int K = g->nk;
    for (int q = 0; q < g->nq; ++q) {
        const double *a = gin + (long)q * K;
        double *p = out + (long)q * K;
        for (int k = 0; k < K; ++k) {
            if (k < 1 || k > K - 2) { p[k] = 0.0; continue; }
            double tp = tau(g, k + 1), tm = tau(g, k - 1);
            double up = tp > 0.0 ? a[k + 1] / tp : 0.0;
            double um = tm > 0.0 ? a[k - 1] / tm : 0.0;
            p[k] = cd * (up - um);
        }
    }
}

/* Exact transpose: g'_k = (C_D / tau_k) (m_{k-1} p_{k-1} - m_{k+1} p_{k+1}), m_j = [1 <= j <= K-2]. */
void oracle_Dt(const orc_geom *g, const double *pin, double *out)
{
    double dt = 1.0 / g->fs;
    double cd = g->gamma / (8.0 * M_PI * g->c * g->c * dt * dt);
    int K = g->nk;
    for (int q = 0; q < g->nq; ++q) {
        const double *p = pin + (long)q * K;
        double *a = out + (long)q * K;
        for (int k = 0; k < K; ++k) {
            double t = tau(g, k);
            if (!(t > 0.0)) { a[k] = 0.0; continue; }
            double lo = (k - 1 >= 1 && k - 1 <= K - 2) ? p[k - 1] : 0.0;
            double hi = (k + 1 >= 1 && k + 1 <= K - 2) ? p[k + 1] : 0.0;
            a[k] = cd / t * (lo - hi);
        }
    }
}

/* ------------------------------------------------------------------ H = D G and H^T = G^T D^T */

void oracle_H(const orc_geom *g, const double *alpha, double *out, int apply_d)
{
    long M = (long)g->nq * g->nk;
    if (!apply_d) { oracle_G(g, alpha, out); return; }
    double *tmp = (double *)malloc(sizeof(double) * M);
    oracle_G(g, alpha, tmp);
    oracle_D(g, tmp, out);
    free(tmp);
}

void oracle_Ht(const orc_geom *g, const double *y, double *out, int apply_d)
{
    long M = (long)g->nq * g->nk;
    if (!apply_d) { oracle_Gt(g, y, out); return; }
    double *tmp = (double *)malloc(sizeof(double) * M);
    oracle_Dt(g, y, tmp);
    oracle_Gt(g, tmp, out);
    free(tmp);
}

/* ------------------------------------------------------------------ brute force and inspection */

/* Dense G: M[(q*K + k)*N + n] = ds^2 sum_{i,j} w_i psi_n(r_{k,i,j}), with psi_n evaluated from its
 * definition for every node n (no 8-neighbour shortcut).  Tiny grids only. */
void oracle_dense_G(const orc_geom *g, double *M)
{
    long N = (long)g->nx * g->ny * g->nz;
    memset(M, 0, sizeof(double) * N * g->nq * g->nk);
    for (int q = 0; q < g->nq; ++q) {
        double ex[3], ey[3], ez[3], rs, rho, dth, dph;
        const double *rq = g->pos + 3 * q;
        transducer_frame(rq, ex, ey, ez, &rs);
        for (int k = 0; k < g->nk; ++k) {
            double *row = M + ((long)q * g->nk + k) * N;
            int ni = shell_rings(g, rs, k, &rho, &dth);
            for (int i = 0; i < ni; ++i) {
                double th = i * dth;
                int nj = ring_points(g, rho, th, &dph);
                double wi = ring_weight(g, rho, th, nj);
                for (int j = 0; j < nj; ++j) {
                    double P[3];
                    lattice_point(rq, ex, ey, ez, rho, th, j * dph, P);
                    for (int iz = 0; iz < g->nz; ++iz)
                        for (int iy = 0; iy < g->ny; ++iy)
                            for (int ix = 0; ix < g->nx; ++ix) {
                                double xn = g->origin[0] + g->ds * ix;
                                double yn = g->origin[1] + g->ds * iy;
                                double zn = g->origin[2] + g->ds * iz;
                                double ax = fabs(P[0] - xn), ay = fabs(P[1] - yn), az = fabs(P[2] - zn);
                                if (ax <= g->ds && ay <= g->ds && az <= g->ds)
                                    row[((long)iz * g->ny + iy) * g->nx + ix] +=
                                        wi * g->ds * g->ds * (1.0 - ax / g->ds) * (1.0 - ay / g->ds) * (1.0 - az / g->ds);
                            }
                }
            }
        }
    }
}

/* Rings and points of one shell: returns the number of points; writes at most cap points
 * (mm, [n][3]), their (i, j) indices and their weights (mm^2). */
long oracle_shell_points(const orc_geom *g, int q, int k, double *P, int *ij, double *wts, long cap, int *n_rings)
{
    double ex[3], ey[3], ez[3], rs, rho, dth, dph;
    const double *rq = g->pos + 3 * q;
    transducer_frame(rq, ex, ey, ez, &rs);
    int ni = shell_rings(g, rs, k, &rho, &dth);
    if (n_rings) *n_rings = ni;
    long n = 0;
    for (int i = 0; i < ni; ++i) {
        double th = i * dth;
        int nj = ring_points(g, rho, th, &dph);
        double wi = ring_weight(g, rho, th, nj) * g->ds * g->ds;
        for (int j = 0; j < nj; ++j, ++n) {
            if (n < cap) {
                if (P) lattice_point(rq, ex, ey, ez, rho, th, j * dph, P + 3 * n);
                if (ij) { ij[2 * n] = i; ij[2 * n + 1] = j; }
                if (wts) wts[n] = wi;
            }
        }
    }
    return n;
}

/* Lattice points of all (q, k): in the support sphere (all) and with at least one of their
 * eight interpolation nodes inside the grid ("useful" points). */
void oracle_count_points(const orc_geom *g, long long *n_ball, long long *n_grid)
{
    long long nb = 0, ng = 0;
    #pragma omp parallel for schedule(dynamic, 1) reduction(+:nb, ng)
    for (int q = 0; q < g->nq; ++q) {
        double ex[3], ey[3], ez[3], rs, rho, dth, dph;
        const double *rq = g->pos + 3 * q;
        transducer_frame(rq, ex, ey, ez, &rs);
        for (int k = 0; k < g->nk; ++k) {
            int ni = shell_rings(g, rs, k, &rho, &dth);
            for (int i = 0; i < ni; ++i) {
                double th = i * dth;
                int nj = ring_points(g, rho, th, &dph);
                for (int j = 0; j < nj; ++j) {
                    double P[3];
                    lattice_point(rq, ex, ey, ez, rho, th, j * dph, P);
                    nb++;
                    double x = (P[0] - g->origin[0]) / g->ds;
                    double y = (P[1] - g->origin[1]) / g->ds;
                    double z = (P[2] - g->origin[2]) / g->ds;
                    if (x >= -1.0 && x < g->nx && y >= -1.0 && y < g->ny && z >= -1.0 && z < g->nz) ng++;
                }
            }
        }
    }
    *n_ball = nb; *n_grid = ng;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
