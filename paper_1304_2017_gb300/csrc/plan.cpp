// Host side of a plan: validation, the FP64 shell-lattice tables (Appendix), the brick tilings
// and device upload.  Compiled without floating-point contraction so that the integer lattice
// counts N_i and N_j come out of plain IEEE double arithmetic in the paper's formula order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <cstdlib>
#include <new>

#include "oat_internal.h"

namespace oat {

namespace {

// v = hi + lo with hi = fl32(v) and lo = fl32(v - hi): a float pair carrying about 48 bits of v.
void split(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

bool finite3(const double *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

// Radius of the origin-centred sphere containing the node cuboid grown by one spacing.
double default_support_radius(const oat_geometry &g) {
    double best = 0.0;
    const double lo[3] = {g.origin_mm[0] - g.spacing_mm, g.origin_mm[1] - g.spacing_mm, g.origin_mm[2] - g.spacing_mm};
    const double hi[3] = {g.origin_mm[0] + g.spacing_mm * g.nx, g.origin_mm[1] + g.spacing_mm * g.ny,
                          g.origin_mm[2] + g.spacing_mm * g.nz};
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                double x = a ? hi[0] : lo[0], y = b ? hi[1] : lo[1], z = c ? hi[2] : lo[2];
                best = std::max(best, std::sqrt(x * x + y * y + z * z));
            }
    return best;
}

// Local frame of a transducer at r (Appendix): e_z towards the origin, e_y = unit(z x r),
// or (0,1,0) on the z axis, e_x = e_y x e_z.
void frame(const double *r, double ex[3], double ey[3], double ez[3], double *rs) {
    double n = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    *rs = n;
    ez[0] = -r[0] / n; ez[1] = -r[1] / n; ez[2] = -r[2] / n;
    double a = -r[1] / n, b = r[0] / n;
    double m = std::sqrt(a * a + b * b);
    if (m > 0.0) { ey[0] = a / m; ey[1] = b / m; ey[2] = 0.0; }
    else { ey[0] = 0.0; ey[1] = 1.0; ey[2] = 0.0; }
    ex[0] = ey[1] * ez[2] - ey[2] * ez[1];
    ex[1] = ey[2] * ez[0] - ey[0] * ez[2];
    ex[2] = ey[0] * ez[1] - ey[1] * ez[0];
}

template <class T>
size_t push_bytes(std::vector<unsigned char> &blob, const std::vector<T> &v) {
    size_t off = (blob.size() + 255) & ~size_t(255);
    blob.resize(off + v.size() * sizeof(T));
    if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
    return off;
}

}  // namespace

int plan_create(const oat_geometry *gin, int device, Plan **out) {
    *out = nullptr;
    if (!gin) return set_error(OAT_ERR_INVALID_ARG, "oat_plan_create: geometry is NULL");
    const oat_geometry &g = *gin;
    if (g.nx < 1 || g.ny < 1 || g.nz < 1)
        return set_error(OAT_ERR_INVALID_ARG, "oat_plan_create: nx, ny, nz must be >= 1");
    if ((long long)g.nx * g.ny * g.nz >= (1LL << 31) ||
        (long long)(g.nx + 1) * (g.ny + 1) * (g.nz + 1) * 8 >= (1LL << 31))
        return set_error(OAT_ERR_INVALID_ARG, "oat_plan_create: grid too large (nx*ny*nz must stay below 2^28)");
    if (g.n_transducers < 1 || !g.positions_mm)
        return set_error(OAT_ERR_INVALID_ARG, "oat_plan_create: need n_transducers >= 1 and positions_mm");
    if (g.n_samples < 1 || (g.apply_d && g.n_samples < 3))
        return set_error(OAT_ERR_INVALID_ARG, "oat_plan_create: n_samples must be >= 1 (>= 3 with apply_d)");
    if ((long long)g.n_transducers * g.n_samples >= (1LL << 31))
        return set_error(OAT_ERR_INVALID_ARG, "oat_plan_create: n_transducers * n_samples must be < 2^31");
    if (!(std::isfinite(g.spacing_mm) && g.spacing_mm > 0) || !(std::isfinite(g.fs_mhz) && g.fs_mhz > 0) ||
        !(std::isfinite(g.c_mm_per_us) && g.c_mm_per_us > 0) || !(std::isfinite(g.t_min_us) && g.t_min_us >= 0) ||
        !std::isfinite(g.support_radius_mm) || !std::isfinite(g.gruneisen) || !finite3(g.origin_mm))
        return set_error(OAT_ERR_INVALID_ARG, "oat_plan_create: spacing, fs, c must be finite and > 0, t_min >= 0, "
                                              "support radius, gruneisen and origin finite");
    if (g.data_dtype != OAT_F32 && g.data_dtype != OAT_F16 && g.data_dtype != OAT_BF16)
        return set_error(OAT_ERR_INVALID_ARG, "oat_plan_create: data_dtype must be OAT_F32, OAT_F16 or OAT_BF16");
    if (g.apply_d != 0 && g.apply_d != 1)
        return set_error(OAT_ERR_INVALID_ARG, "oat_plan_create: apply_d must be 0 or 1");
    if (g.lattice_weights != OAT_LATTICE_UNIFORM && g.lattice_weights != OAT_LATTICE_EXACT_AREA)
        return set_error(OAT_ERR_INVALID_ARG, "oat_plan_create: lattice_weights must be OAT_LATTICE_UNIFORM or OAT_LATTICE_EXACT_AREA");

    Plan *p = new (std::nothrow) Plan();
    if (!p) return set_error(OAT_ERR_OOM, "oat_plan_create: host allocation failed");
    p->g = g;
    p->Q = g.n_transducers; p->K = g.n_samples;
    p->nx = g.nx; p->ny = g.ny; p->nz = g.nz;
    p->pos.assign(g.positions_mm, g.positions_mm + 3 * (size_t)p->Q);
    p->g.positions_mm = p->pos.data();
    p->device = device;
    for (int q = 0; q < p->Q; ++q)
        if (!finite3(&p->pos[3 * q])) { delete p; return set_error(OAT_ERR_INVALID_ARG, "oat_plan_create: non-finite transducer position"); }

    p->R = g.support_radius_mm > 0 ? g.support_radius_mm : default_support_radius(g);
    p->dt = 1.0 / g.fs_mhz;
    p->cd = g.gruneisen / (8.0 * M_PI * g.c_mm_per_us * g.c_mm_per_us * p->dt * p->dt);
    const double ds = g.spacing_mm;
    for (int d = 0; d < 3; ++d) split(-g.origin_mm[d] / ds, p->O[d], p->O_lo[d]);
    p->ds2 = (float)(ds * ds);
    p->R0 = (float)(g.c_mm_per_us * g.t_min_us / ds);
    p->dR = (float)(g.c_mm_per_us * p->dt / ds);

    // transducers: frames and radius classes (exact equality of |r_q| in double)
    const int Q = p->Q, K = p->K;
    std::vector<Xdcr> xd(Q);
    std::vector<double> rs(Q);
    std::map<double, int> cls_of;
    for (int q = 0; q < Q; ++q) {
        double ex[3], ey[3], ez[3];
        frame(&p->pos[3 * q], ex, ey, ez, &rs[q]);
        if (!(rs[q] > p->R)) {
            delete p;
            return set_error(OAT_ERR_GEOMETRY, "oat_plan_create: transducer " + std::to_string(q) +
                                                   " is not outside the support sphere (|r_q| <= R)");
        }
        for (int d = 0; d < 3; ++d) {
            split(ex[d], xd[q].ex[d], xd[q].ex_lo[d]);
            split(ey[d], xd[q].ey[d], xd[q].ey_lo[d]);
            split(ez[d], xd[q].ez[d], xd[q].ez_lo[d]);
        }
        xd[q].dist = (float)(rs[q] / ds);
        cls_of.emplace(rs[q], 0);
    }
    std::vector<double> cls_r;
    for (auto &kv : cls_of) { kv.second = (int)cls_r.size(); cls_r.push_back(kv.first); }
    p->n_cls = (int)cls_r.size();
    for (int q = 0; q < Q; ++q) xd[q].cls = cls_of[rs[q]];

    // shell lattice per (class, k): rings i < N_i with N_j points each, and the anchors of every
    // ring: points j = t 2^ash, local coordinates a (cos(j dphi), sin(j dphi)) as float pairs
    const int C = p->n_cls;
    std::vector<Ring> rings;
    std::vector<float> ring_w;          // exact strip areas: point weight / Delta_s^2 per ring
    std::vector<float4> anchors;
    const bool area = g.lattice_weights == OAT_LATTICE_EXACT_AREA;
    double wsum_max = 0.0, wring_max = 0.0;
    std::vector<int> ring_off((size_t)C * K), ring_cnt((size_t)C * K);
    p->cls_points.assign((size_t)C * K, 0);
    for (int c = 0; c < C; ++c) {
        const double r_s = cls_r[c];
        for (int k = 0; k < K; ++k) {
            const size_t ck = (size_t)c * K + k;
            ring_off[ck] = (int)rings.size();
            ring_cnt[ck] = 0;
            double t = g.t_min_us + k * p->dt;
            double rho = g.c_mm_per_us * t;
            if (!(rho > 0.0)) continue;
            double arg = (r_s * r_s + rho * rho - p->R * p->R) / (2.0 * rho * r_s);
            if (arg > 1.0) continue;
            double thmax = (arg < -1.0) ? M_PI : std::acos(arg);
            double dth = ds / rho;
            int ni = (int)std::floor(thmax / dth);
            if (rings.size() + (size_t)ni >= (size_t)INT32_MAX) {
                delete p;
                return set_error(OAT_ERR_UNSUPPORTED, "oat_plan_create: lattice tables exceed 2^31 rings");
            }
            long long npts = 0;
            double wsum = 0.0;
            for (int i = 0; i < ni; ++i) {
                double th = i * dth;
                double st = std::sin(th);
                double dph = ds / (rho * st);
                int nj = (int)std::floor(2.0 * M_PI / dph);
                const double h = (rho * std::cos(th) - r_s) / ds, a = rho * st / ds;
                Ring rr;
                split(h, rr.h, rr.h_lo);
                rr.a = (float)a;
                split(dph, rr.dphi, rr.dphi_lo);
                rr.nj = nj;
                // anchors every 2^ash points, the longest run whose rotation stays within 1 rad
                int ash = kMaxAnchorShift;
                while (ash > 0 && (double)(1 << ash) * dph > 1.0) --ash;
                rr.ash = ash;
                rr.aoff = (int)anchors.size();
                if (nj == 0) { rr.dphi = 0.f; rr.dphi_lo = 0.f; rr.a = 0.f; rr.ash = kMaxAnchorShift; }
                const int na = nj > 0 ? ((nj + (1 << rr.ash) - 1) >> rr.ash) : 0;
                if (anchors.size() + (size_t)na >= (size_t)INT32_MAX) {
                    delete p;
                    return set_error(OAT_ERR_UNSUPPORTED, "oat_plan_create: lattice tables exceed 2^31 anchors");
                }
                for (int tt = 0; tt < na; ++tt) {
                    const double phi = (double)(tt << rr.ash) * dph;
                    float4 e;
                    split(a * std::cos(phi), e.x, e.y);
                    split(a * std::sin(phi), e.z, e.w);
                    anchors.push_back(e);
                }
                rings.push_back(rr);
                npts += nj;
                if (area) {
                    // the strip of ring i (polar width dtheta, i.e. Delta_s on the shell; length
                    // 2 pi rho sin theta_i) shared by its N_j points, over Delta_s^2
                    const double wi = nj > 0 ? 2.0 * M_PI * a / nj : 0.0;
                    ring_w.push_back((float)wi);
                    wsum += (double)(float)wi * nj;
                    wring_max = std::max(wring_max, (double)(float)wi);
                }
            }
            wsum_max = std::max(wsum_max, wsum);
            ring_cnt[ck] = ni;
            p->cls_points[ck] = npts;
        }
    }
    p->n_rings = (long long)rings.size();
    p->n_anchors = (long long)anchors.size();

    std::vector<int> cls_n(C, 0);
    for (int q = 0; q < Q; ++q) cls_n[xd[q].cls]++;
    p->points_ball = 0;
    for (int c = 0; c < C; ++c)
        for (int k = 0; k < K; ++k) p->points_ball += p->cls_points[(size_t)c * K + k] * cls_n[c];
    if (p->points_ball == 0) {
        delete p;
        return set_error(OAT_ERR_GEOMETRY, "oat_plan_create: no shell of the time window meets the support sphere");
    }

    p->max_shell_points = 0;
    for (long long np : p->cls_points) p->max_shell_points = std::max(p->max_shell_points, np);
    // bound of |G alpha| / max|alpha| in units of Delta_s^2 (the projector's fixed-point range)
    p->area = area;
    p->fwd_bound = area ? wsum_max * (1.0 + 1e-6) : (double)p->max_shell_points;

    {
        // grid sizes follow the device's SM count (the first device call: host validation is done)
        cudaError_t ea = cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, device);
        if (ea != cudaSuccess || p->n_sm < 1) {
            delete p;
            cudaGetLastError();
            return set_error(OAT_ERR_CUDA, std::string("oat_plan_create: cudaDeviceGetAttribute(SM count): ") +
                                               cudaGetErrorString(ea));
        }
    }
    // brick tilings of the cells [-1, n-1] for the two directions
    auto tile = [&](BrickCfg &bc, int B, size_t node_bytes) {
        const int n[3] = {p->nx, p->ny, p->nz};
        long long bricks = 1;
        double diag2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            bc.nb[d] = (n[d] + 1 + B - 1) / B;
            bc.bs[d] = (n[d] + 1 + bc.nb[d] - 1) / bc.nb[d];
            while (bc.nb[d] > 1 && bc.bs[d] * (bc.nb[d] - 1) >= n[d] + 1) --bc.nb[d];   // no empty brick
            bricks *= bc.nb[d];
            diag2 += (double)bc.bs[d] * bc.bs[d];
        }
        const double rb = 0.5 * std::sqrt(diag2) + 0.05;
        bc.kspan = (int)std::ceil(2.0 * rb / (g.c_mm_per_us * p->dt / ds)) + 2;
        // transducer chunks per brick: at least 8 work items per SM, and as few chunks as leave at
        // most 2 % of the last wave of work items idle (one block per SM at a time)
        const long long sms = p->n_sm;
        const long long c0 = std::max(1LL, std::min<long long>(Q, (sms * 8 + bricks - 1) / bricks));
        auto items_of = [&](long long c) {
            const long long qc = (Q + c - 1) / c;
            return bricks * ((Q + qc - 1) / qc);
        };
        auto waste = [&](long long c) {
            const long long it = items_of(c);
            return (double)(((it + sms - 1) / sms) * sms) / (double)it - 1.0;
        };
        long long chunks = c0;
        for (long long c = c0; c <= std::min<long long>(Q, 8 * c0); ++c) {
            if (waste(c) <= 0.02) { chunks = c; break; }
            if (waste(c) < waste(chunks)) chunks = c;
        }
        bc.qchunk = (int)((Q + chunks - 1) / chunks);
        bc.items = items_of(chunks);
        bc.smem = node_bytes * (size_t)(B + 1) * (B + 1) * (B + 1);
    };
    tile(p->fwd, kBF, sizeof(float));
    p->fwd.smem = forward_smem_bytes();
    tile(p->adj, kBA, 2 * sizeof(int));
    p->adj.smem = adjoint_smem_bytes(area);
    {
        // contributions one transducer adds to one node: 8 cells x (shells crossing a cell:
        // diameter sqrt(3) over the shell spacing, + 2) x (2 rings x 3 points, + margin)
        const double dRs = g.c_mm_per_us * p->dt / ds;
        const long long shells = (long long)std::floor(std::sqrt(3.0) / dRs) + 2;
        const long long per_q = 8 * shells * 9;
        p->adj_qpass = (int)std::max<long long>(1, std::min<long long>(Q, 32768 / per_q));
        if (per_q > 32768) {
            delete p;
            return set_error(OAT_ERR_UNSUPPORTED, "oat_plan_create: shells too dense for the backprojector's "
                                                  "fixed-point accumulation (c dt / spacing too small)");
        }
        // the volume accumulator's unit: a node receives at most per_q Q contributions of at
        // most 2^adj_fbits units each, which must stay below 2^62 in magnitude
        int lb = 0;
        while ((1LL << lb) < per_q * (long long)Q) ++lb;
        p->adj_fbits = 62 - lb;
    }

    std::vector<float> Rk(K), wD(K);
    std::vector<double> wD64(K);
    for (int k = 0; k < K; ++k) {
        double t = g.t_min_us + k * p->dt;
        Rk[k] = (float)(g.c_mm_per_us * t / ds);
        double tau = g.t_min_us / p->dt + k;
        wD[k] = tau > 0.0 ? (float)(p->cd / tau) : 0.f;
        wD64[k] = tau > 0.0 ? p->cd / tau : 0.0;
    }
    // G^T: a point's weight factor is at most wring_max with exact strip areas (1 otherwise)
    p->adj_wfac = area ? (float)(wring_max * (1.0 + 1e-6)) : 1.f;

    // per transducer, the samples whose shells can hold a point in a cell of the grid (the node
    // box grown by one spacing, the trilinear support), with two samples of margin: the
    // backprojector bounds g' over these only
    std::vector<int2> krange(Q);
    {
        const double lo[3] = {g.origin_mm[0] - ds, g.origin_mm[1] - ds, g.origin_mm[2] - ds};
        const double hi[3] = {g.origin_mm[0] + ds * g.nx, g.origin_mm[1] + ds * g.ny, g.origin_mm[2] + ds * g.nz};
        for (int q = 0; q < Q; ++q) {
            double dn = 0.0, df = 0.0;
            for (int d = 0; d < 3; ++d) {
                const double x = p->pos[3 * q + d];
                const double near = x < lo[d] ? lo[d] - x : (x > hi[d] ? x - hi[d] : 0.0);
                const double far = std::max(std::fabs(x - lo[d]), std::fabs(x - hi[d]));
                dn += near * near;
                df += far * far;
            }
            const double k0 = std::floor((std::sqrt(dn) / g.c_mm_per_us - g.t_min_us) / p->dt) - 2.0;
            const double k1 = std::ceil((std::sqrt(df) / g.c_mm_per_us - g.t_min_us) / p->dt) + 2.0;
            const int a = (int)std::max(0.0, std::min((double)K, k0));
            const int b = (int)std::max(-1.0, std::min((double)K - 1, k1));
            krange[q] = make_int2(a, b);   // empty when a > b
        }
    }

    // one device blob for every table
    std::vector<unsigned char> blob;
    size_t o_rings = push_bytes(blob, rings), o_off = push_bytes(blob, ring_off), o_cnt = push_bytes(blob, ring_cnt);
    size_t o_xd = push_bytes(blob, xd), o_an = push_bytes(blob, anchors);
    size_t o_rk = push_bytes(blob, Rk), o_wd = push_bytes(blob, wD), o_wd64 = push_bytes(blob, wD64);
    size_t o_rw = push_bytes(blob, ring_w);
    size_t o_kr = push_bytes(blob, krange);
    std::vector<float4>().swap(anchors);
    p->table_bytes = (long long)blob.size();

    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete p;
        return set_error(OAT_ERR_CUDA, std::string("oat_plan_create: cudaSetDevice: ") + cudaGetErrorString(e));
    }
    auto fail = [&](cudaError_t err, const char *what) {
        int code = (err == cudaErrorMemoryAllocation) ? OAT_ERR_OOM : OAT_ERR_CUDA;
        if (p->d_tables) cudaFree(p->d_tables);
        if (p->d_gacc) cudaFree(p->d_gacc);
        if (p->d_vacc) cudaFree(p->d_vacc);
        if (p->d_amax) cudaFree(p->d_amax);
        if (p->d_rowmax) cudaFree(p->d_rowmax);
        if (p->d_fbp) cudaFree(p->d_fbp);
        delete p;
        cudaGetLastError();
        cudaSetDevice(prev);
        return set_error(code, std::string("oat_plan_create: ") + what + ": " + cudaGetErrorString(err));
    };
    if ((e = cudaMalloc(&p->d_tables, blob.size())) != cudaSuccess) return fail(e, "cudaMalloc(tables)");
    if ((e = cudaMemcpy(p->d_tables, blob.data(), blob.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "cudaMemcpy(tables)");
    size_t g_bytes = sizeof(long long) * (size_t)Q * K;
    size_t v_bytes = sizeof(long long) * (size_t)p->nx * p->ny * p->nz;
    if ((e = cudaMalloc(&p->d_gacc, g_bytes)) != cudaSuccess) return fail(e, "cudaMalloc(G scratch)");
    if ((e = cudaMalloc(&p->d_vacc, v_bytes)) != cudaSuccess) return fail(e, "cudaMalloc(G^T scratch)");
    if ((e = cudaMalloc(&p->d_amax, 256)) != cudaSuccess) return fail(e, "cudaMalloc(scale scratch)");
    if ((e = cudaMalloc(&p->d_rowmax, sizeof(float) * (size_t)Q)) != cudaSuccess) return fail(e, "cudaMalloc(row maxima)");
    // FBP table: transducer positions in index units as float pairs; weights set later
    p->fbp_host.resize(2 * (size_t)Q);
    for (int q = 0; q < Q; ++q) {
        float hi[3], lo[3];
        for (int d = 0; d < 3; ++d) split((p->pos[3 * q + d] - g.origin_mm[d]) / ds, hi[d], lo[d]);
        p->fbp_host[2 * q] = make_float4(hi[0], hi[1], hi[2], 0.f);
        p->fbp_host[2 * q + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
    }
    if ((e = cudaMalloc(&p->d_fbp, sizeof(float4) * p->fbp_host.size())) != cudaSuccess) return fail(e, "cudaMalloc(FBP table)");
    if ((e = cudaMemcpy(p->d_fbp, p->fbp_host.data(), sizeof(float4) * p->fbp_host.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return fail(e, "cudaMemcpy(FBP table)");
    p->d_count = (unsigned long long *)((char *)p->d_amax + 128);
    p->scratch_bytes = (long long)(g_bytes + v_bytes + 256 + sizeof(float) * (size_t)Q + sizeof(float4) * p->fbp_host.size());
    if (set_forward_attributes() != OAT_OK || set_adjoint_attributes() != OAT_OK) {
        std::string msg = std::string("oat_plan_create: ") + oat_last_error();
        fail(cudaSuccess, "kernel attributes");
        return set_error(OAT_ERR_CUDA, msg);
    }
    cudaSetDevice(prev);

    unsigned char *base = (unsigned char *)p->d_tables;
    p->t.rings = (const Ring *)(base + o_rings);
    p->t.ring_off = (const int *)(base + o_off);
    p->t.ring_cnt = (const int *)(base + o_cnt);
    p->t.xd = (const Xdcr *)(base + o_xd);
    p->t.anchors = (const float4 *)(base + o_an);
    p->t.Rk = (const float *)(base + o_rk);
    p->t.wD = (const float *)(base + o_wd);
    p->t.wD64 = (const double *)(base + o_wd64);
    p->t.ring_w = area ? (const float *)(base + o_rw) : nullptr;
    p->d_krange = (const int2 *)(base + o_kr);
    *out = p;
    return OAT_OK;
}

void plan_destroy(Plan *p) {
    if (!p) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    for (int w = 0; w < 3; ++w)
        for (cudaEvent_t e : p->ev[w]) cudaEventDestroy(e);
    if (p->d_tables) cudaFree(p->d_tables);
    if (p->d_fbp) cudaFree(p->d_fbp);
    if (p->d_gacc) cudaFree(p->d_gacc);
    if (p->d_vacc) cudaFree(p->d_vacc);
    if (p->d_amax) cudaFree(p->d_amax);
    if (p->d_rowmax) cudaFree(p->d_rowmax);
    if (p->d_eir) cudaFree(p->d_eir);
    if (p->d_eir_z) cudaFree(p->d_eir_z);
    cudaSetDevice(prev);
    delete p;
}

}  // namespace oat
