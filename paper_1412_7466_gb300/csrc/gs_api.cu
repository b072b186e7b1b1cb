// C-ABI entry points of the gsolve library: context, problem definition, factorisation, and the
// hot-path calls (translate, apply, rhs, solve, Bragg).  Host code validates arguments, owns the
// device buffers and orchestrates kernels on the context's stream; all arithmetic of the method
// runs in the CUDA kernels of gs_assemble.cu, gs_svd.cu, gs_translate.cu and gs_solve.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gs_internal.h"

size_t gs_translate_scratch_elems(int M, int p);

int gs_fail(gs_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

bool gs_prof_pair(gs_ctx *c, cudaEvent_t *e0, cudaEvent_t *e1, int precision) {
    if (!c->prof_on) return false;
    while (c->prof_ev.size() < c->prof_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        c->prof_ev.push_back(e);
    }
    *e0 = c->prof_ev[c->prof_used];
    *e1 = c->prof_ev[c->prof_used + 1];
    if (c->prof_prec.size() < c->prof_used / 2 + 1) c->prof_prec.resize(c->prof_used / 2 + 1);
    c->prof_prec[c->prof_used / 2] = precision;
    c->prof_used += 2;
    return true;
}

namespace {

template <typename T>
int dalloc(gs_ctx *c, T **p, size_t n) {
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
    }
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * n);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return gs_fail(c, GS_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(sizeof(T) * n) +
                                          " bytes: " + cudaGetErrorString(e));
    }
    return GS_OK;
}
template <typename T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// geometry-dependent data of an angle (rebuilt by gs_factor after gs_set_inclusions)
void free_angle_geometry(AngleData &a) {
    dfree(a.B);
    dfree(a.Cm);
    dfree(a.B32);
    dfree(a.C2);
    a.C2_off = false;
    a.C2_ready = false;
    dfree(a.beta);
    a.iters = 0;
    a.outer = 0;
    a.relres = -1.0;
}

void free_angle(AngleData &a) {
    dfree(a.kappa);
    dfree(a.k1n);
    dfree(a.k3n);
    dfree(a.f);
    dfree(a.W);
    dfree(a.Vr);
    dfree(a.dscale);
    dfree(a.coef);
    dfree(a.sigma);
    dfree(a.WH2);
    dfree(a.Vr2);
    a.A2_off = false;
    a.A2_ready = false;
    free_angle_geometry(a);
}

// everything sized by the number of unknowns n = M (2p+1)
void free_geometry(gs_ctx *c) {
    for (auto &a : c->ang) free_angle_geometry(a);
    dfree(c->v1);
    dfree(c->v2);
    dfree(c->v3);
    dfree(c->v4);
    dfree(c->v5);
    dfree(c->v6);
    dfree(c->part);
    dfree(c->b32);
    dfree(c->img32);
    dfree(c->xdf);
    dfree(c->adf);
    c->adf_n = 0;
    dfree(c->iflag);
    dfree(c->htab);
    dfree(c->tab32.h);
    c->tab32.sp = 0;
    c->tab32_off = false;
    dfree(c->b3pad);
    gs_angles_destroy(c);
    if (c->tcA) cudaFree(c->tcA);
    c->tcA = nullptr;
    for (int q = 0; q < 2; ++q) {
        if (c->tcA_sp[q]) cudaFree(c->tcA_sp[q]);
        c->tcA_sp[q] = nullptr;
    }
    c->tcA_rows = c->tcA_cols = 0;
    if (c->sp_scratch) cudaFree(c->sp_scratch);
    c->sp_scratch = nullptr;
    c->sp_scratch_bytes = 0;
    c->sp_zeroed_R = -1;
    if (c->tc_scratch) cudaFree(c->tc_scratch);
    c->tc_scratch = nullptr;
    c->tc_scratch_bytes = 0;
    c->tc_zeroed_rp = c->tc_zeroed_k = c->tc_zeroed_R = -1;
    c->part_elems = 0;
    dfree(c->Vk);
    dfree(c->kv1);
    dfree(c->kv2);
    dfree(c->Hh);
    dfree(c->cs);
    dfree(c->sn);
    dfree(c->gg);
    dfree(c->yy);
    dfree(c->kw32);
    dfree(c->dpart);
    dfree(c->npart);
    c->kdim = 0;
    c->factored = false;
}

// everything, including the per-angle factorisation of the empty grating; the batch too unless
// keep_batch (rebuilding the grating factorisation for a batch must not discard that batch)
void free_factor(gs_ctx *c, bool keep_batch = false) {
    if (!keep_batch) gs_batch_destroy(c);
    free_geometry(c);
    for (auto &a : c->ang) free_angle(a);
    c->ang.clear();
    dfree(c->g);
    dfree(c->w);
    dfree(c->x);
    dfree(c->x32);
    dfree(c->Vtmp);
    dfree(c->Xtmp);
    dfree(c->Vxtmp);
    dfree(c->X32tmp);
    dfree(c->nrm2);
    dfree(c->perm);
    dfree(c->tau);
    c->grating_ready = false;
}

double iface_h(const gs_ctx *c, int which, double x) {
    const gs_layers &L = c->L;
    double h = which == 0 ? L.h1_0 : L.h2_0;
    const std::vector<double> &ca = c->four[2 * which], &sa = c->four[2 * which + 1];
    for (int m = 1; m <= L.n_fourier; ++m) {
        double om = 2.0 * M_PI * m / L.d;
        h += ca[m - 1] * std::cos(om * x) + sa[m - 1] * std::sin(om * x);
    }
    return h;
}

bool in_range(int v, int lo, int hi) { return v >= lo && v <= hi; }

#define CTX_GUARD(c)                                   \
    do {                                               \
        if (!(c)) return GS_ERR_ARG;                   \
        cudaError_t e_ = cudaSetDevice((c)->device);   \
        if (e_ != cudaSuccess) return gs_fail((c), GS_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)

int check_angle(gs_ctx *c, int angle) {
    if (!c->factored) return gs_fail(c, GS_ERR_STATE, "gs_factor has not run");
    if (angle < 0 || angle >= (int)c->ang.size()) return gs_fail(c, GS_ERR_ARG, "angle index out of range");
    return GS_OK;
}

}  // namespace

// Krylov workspace of the single-geometry solve for a restart length of up to 512
int gs_ensure_krylov(gs_ctx *c, int restart) {
    const int want = std::max(1, std::min(restart, 512));
    const long n = c->n();
    if (!c->kw32) GS_TRY(dalloc(c, &c->kw32, n));
    if (!c->dpart) GS_TRY(dalloc(c, &c->dpart, (size_t)GS_DOT_SPLIT * 513));
    if (!c->npart) GS_TRY(dalloc(c, &c->npart, GS_NORM_PARTS));
    if (c->Vk && c->kdim >= want) return GS_OK;
    c->kdim = want;
    GS_TRY(dalloc(c, &c->Vk, (size_t)(c->kdim + 1) * n));
    GS_TRY(dalloc(c, &c->kv1, n));
    GS_TRY(dalloc(c, &c->kv2, n));
    GS_TRY(dalloc(c, &c->Hh, (size_t)(c->kdim + 1) * c->kdim));
    GS_TRY(dalloc(c, &c->cs, c->kdim + 1));
    GS_TRY(dalloc(c, &c->sn, c->kdim + 1));
    GS_TRY(dalloc(c, &c->gg, c->kdim + 1));
    GS_TRY(dalloc(c, &c->yy, c->kdim + 1));
    return GS_OK;
}

int gs_ensure_grating(gs_ctx *c) {
    const Layout &ly = c->lay;
    // per-angle factorisation of the empty grating (kept across gs_set_inclusions)
    if (!c->grating_ready) {
        free_factor(c, true);
        GS_TRY(dalloc(c, &c->g, ly.rows));
        GS_TRY(dalloc(c, &c->w, ly.cols));
        GS_TRY(dalloc(c, &c->x, ly.cols));
        GS_TRY(dalloc(c, &c->x32, ly.cols));
        GS_TRY(dalloc(c, &c->Vtmp, (size_t)ly.rows * ly.cols));
        GS_TRY(dalloc(c, &c->Xtmp, (size_t)ly.cols * ly.cols));
        GS_TRY(dalloc(c, &c->Vxtmp, (size_t)ly.cols * ly.cols));
        GS_TRY(dalloc(c, &c->X32tmp, 2 * (size_t)ly.cols * ly.cols));
        GS_TRY(dalloc(c, &c->nrm2, ly.cols));
        GS_TRY(dalloc(c, &c->perm, ly.cols));
        GS_TRY(dalloc(c, &c->tau, ly.cols));
        c->ang.resize(c->thetas.size());
        for (size_t q = 0; q < c->thetas.size(); ++q) {
            AngleData &a = c->ang[q];
            a.theta = c->thetas[q];
            int K2 = 2 * ly.K + 1;
            GS_TRY(dalloc(c, &a.kappa, K2));
            GS_TRY(dalloc(c, &a.k1n, K2));
            GS_TRY(dalloc(c, &a.k3n, K2));
            GS_TRY(dalloc(c, &a.f, ly.rows));
            GS_TRY(dalloc(c, &a.W, (size_t)ly.rows * ly.cols));
            GS_TRY(dalloc(c, &a.Vr, (size_t)ly.cols * ly.cols));
            GS_TRY(dalloc(c, &a.dscale, ly.cols));
            GS_TRY(dalloc(c, &a.coef, ly.cols));
            GS_TRY(dalloc(c, &a.sigma, ly.cols));
            GS_TRY(gs_angle_scalars(c, a));
            GS_TRY(gs_factor_angle(c, a));
        }
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
        dfree(c->Vtmp);
        dfree(c->Xtmp);
        dfree(c->Vxtmp);
        dfree(c->X32tmp);
        c->grating_ready = true;
    }
    return GS_OK;
}

extern "C" {

const char *gs_strerror(int s) {
    switch (s) {
        case GS_OK: return "ok";
        case GS_ERR_ARG: return "invalid argument";
        case GS_ERR_STATE: return "call out of order";
        case GS_ERR_CUDA: return "CUDA error";
        case GS_ERR_OOM: return "out of device memory";
        case GS_ERR_GEOMETRY: return "invalid geometry";
        case GS_ERR_NOT_CONVERGED: return "GMRES did not converge";
        case GS_ERR_NUMERIC: return "non-finite result";
        case GS_ERR_TIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char *gs_last_error(gs_ctx *c) { return c ? c->err.c_str() : "null context"; }

int gs_create(gs_ctx **out, int device, void *cuda_stream) {
    if (!out) return GS_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return GS_ERR_CUDA;
    gs_ctx *c = new gs_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || c->sms < 1) {
        cudaGetLastError();
        delete c;
        return GS_ERR_CUDA;
    }
    if (cudaMalloc((void **)&c->dscal, sizeof(double) * 16) != cudaSuccess ||
        cudaMallocHost((void **)&c->hscal, sizeof(double) * 16) != cudaSuccess ||
        cudaMalloc((void **)&c->dcount, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void **)&c->terr, sizeof(int)) != cudaSuccess || cudaMemset(c->terr, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void **)&c->bar, 2 * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        gs_destroy(c);
        return GS_ERR_OOM;
    }
    *out = c;
    return GS_OK;
}

void gs_destroy(gs_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    gs_mlp_destroy(c);
    free_factor(c);
    for (int q = 0; q < 2; ++q) dfree(c->curve[q]);
    for (int q = 0; q < 3; ++q) dfree(c->wall_y[q]);
    dfree(c->bound_x);
    dfree(c->kress);
    dfree(c->four_dev);
    dfree(c->xy);
    dfree(c->radius);
    dfree(c->kp);
    dfree(c->kp_im);
    dfree(c->star_phi);
    dfree(c->S0);
    dfree(c->Sblk);
    dfree(c->s);
    dfree(c->dscal);
    dfree(c->dcount);
    dfree(c->terr);
    dfree(c->bar);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    if (c->hscal) cudaFreeHost(c->hscal);
    delete c;
}

int gs_set_layers(gs_ctx *c, const gs_layers *L) {
    CTX_GUARD(c);
    if (!L) return gs_fail(c, GS_ERR_ARG, "null layers");
    if (!(L->d > 0) || !(L->k1 > 0) || !(L->k2 > 0) || !(L->k3 > 0) || !(L->eps_pinv > 0) || !(L->y0 > 0))
        return gs_fail(c, GS_ERR_ARG, "d, k1, k2, k3, y0 and eps_pinv must be positive");
    if (L->N < 8 || L->N > 4096 || (L->N & 1)) return gs_fail(c, GS_ERR_ARG, "N must be even in [8, 4096]");
    if (!in_range(L->Q1, 1, 1024) || !in_range(L->Q2, 1, 1024) || !in_range(L->Q3, 1, 1024) ||
        !in_range(L->K_rb, 1, 1024) || !in_range(L->n_wall1, 1, 1024) || !in_range(L->n_wall2, 1, 1024) ||
        !in_range(L->n_wall3, 1, 1024) || !in_range(L->n_bound, 1, 1024) || !in_range(L->n_fourier, 0, 64))
        return gs_fail(c, GS_ERR_ARG, "Q, K_rb, n_wall, n_bound must be in [1, 1024], n_fourier in [0, 64]");
    if (L->n_fourier > 0 && (!L->h1_cos || !L->h1_sin || !L->h2_cos || !L->h2_sin))
        return gs_fail(c, GS_ERR_ARG, "null Fourier coefficient array");
    free_factor(c);
    c->L = *L;
    const double *src[4] = {L->h1_cos, L->h1_sin, L->h2_cos, L->h2_sin};
    for (int q = 0; q < 4; ++q) c->four[q].assign(src[q], src[q] + L->n_fourier);
    c->L.h1_cos = c->L.h1_sin = c->L.h2_cos = c->L.h2_sin = nullptr;
    Layout &y = c->lay;
    y.N = L->N;
    y.Q1 = L->Q1;
    y.Q2 = L->Q2;
    y.Q3 = L->Q3;
    y.K = L->K_rb;
    y.nw1 = L->n_wall1;
    y.nw2 = L->n_wall2;
    y.nw3 = L->n_wall3;
    y.nb = L->n_bound;
    int N = L->N;
    y.col_mu1 = 0;
    y.col_sig1 = N;
    y.col_mu2 = 2 * N;
    y.col_sig2 = 3 * N;
    y.col_a2 = 4 * N;
    y.col_a1 = y.col_a2 + 2 * y.Q2 + 1;
    y.col_a3 = y.col_a1 + 2 * y.Q1 + 1;
    y.col_c = y.col_a3 + 2 * y.Q3 + 1;
    y.col_d = y.col_c + 2 * y.K + 1;
    y.cols = y.col_d + 2 * y.K + 1;
    y.row_g1v = 0;
    y.row_g1n = N;
    y.row_g2v = 2 * N;
    y.row_g2n = 3 * N;
    y.row_w2v = 4 * N;
    y.row_w2n = y.row_w2v + y.nw2;
    y.row_w1v = y.row_w2n + y.nw2;
    y.row_w1n = y.row_w1v + y.nw1;
    y.row_w3v = y.row_w1n + y.nw1;
    y.row_w3n = y.row_w3v + y.nw3;
    y.row_uv = y.row_w3n + y.nw3;
    y.row_un = y.row_uv + y.nb;
    y.row_dv = y.row_un + y.nb;
    y.row_dn = y.row_dv + y.nb;
    y.rows = y.row_dn + y.nb;
    if (y.rows < y.cols) return gs_fail(c, GS_ERR_ARG, "A must have at least as many rows as columns");
    c->yL1 = iface_h(c, 0, -0.5 * L->d);
    c->yL2 = iface_h(c, 1, -0.5 * L->d);
    double h1min = 1e300, h2max = -1e300;
    for (int i = 0; i < 4096; ++i) {
        double x = -0.5 * L->d + (i + 0.5) * L->d / 4096;
        h1min = std::min(h1min, iface_h(c, 0, x));
        h2max = std::max(h2max, iface_h(c, 1, x));
    }
    c->h1_min = h1min;
    c->h2_max = h2max;
    if (!(h2max < h1min && L->y0 > c->h1_min)) {
        // the layers must be ordered: Gamma2 below Gamma1 below Gamma_u
        double h1max = -1e300, h2min = 1e300;
        for (int i = 0; i < 4096; ++i) {
            double x = -0.5 * L->d + (i + 0.5) * L->d / 4096;
            h1max = std::max(h1max, iface_h(c, 0, x));
            h2min = std::min(h2min, iface_h(c, 1, x));
        }
        if (!(h2max < h1min) || !(L->y0 > h1max) || !(-L->y0 < h2min))
            return gs_fail(c, GS_ERR_GEOMETRY, "interfaces must satisfy -y0 < Gamma2 < Gamma1 < y0");
    }
    for (int q = 0; q < 2; ++q) GS_TRY(dalloc(c, &c->curve[q], 8 * (size_t)N));
    GS_TRY(dalloc(c, &c->wall_y[0], y.nw1));
    GS_TRY(dalloc(c, &c->wall_y[1], y.nw2));
    GS_TRY(dalloc(c, &c->wall_y[2], y.nw3));
    GS_TRY(dalloc(c, &c->bound_x, y.nb));
    GS_TRY(dalloc(c, &c->kress, N));
    GS_TRY(dalloc(c, &c->four_dev, 4 * (size_t)std::max(1, L->n_fourier)));
    GS_TRY(gs_build_geometry(c));
    c->have_layers = true;
    c->have_inc = false;   // clearance of the disks must be re-validated
    return GS_OK;
}

int gs_set_incidence(gs_ctx *c, int n_angles, const double *theta) {
    CTX_GUARD(c);
    if (n_angles < 1 || n_angles > 4096 || !theta) return gs_fail(c, GS_ERR_ARG, "need 1..4096 angles");
    for (int i = 0; i < n_angles; ++i)
        if (!std::isfinite(theta[i]) || std::sin(theta[i]) >= 0.0)
            return gs_fail(c, GS_ERR_ARG, "incidence must travel downwards (sin(theta) < 0)");
    free_factor(c);
    c->thetas.assign(theta, theta + n_angles);
    return GS_OK;
}

int gs_set_inclusions(gs_ctx *c, const gs_inclusions *I) {
    CTX_GUARD(c);
    if (!I || I->M < 1 || I->M > 1000000 || !I->xy || !I->radius || !I->kp)
        return gs_fail(c, GS_ERR_ARG, "need 1..1e6 disks with xy, radius and kp");
    if (!c->have_layers) return gs_fail(c, GS_ERR_STATE, "gs_set_layers must come first");
    switch (I->p) {
        case 1: case 2: case 3: case 4: case 5: case 6: case 7: case 8: case 10: case 12: case 16: break;
        default: return gs_fail(c, GS_ERR_ARG, "multipole order p must be one of 1-8, 10, 12, 16");
    }
    const double d = c->L.d;
    for (int i = 0; i < I->M; ++i) {
        double x = I->xy[2 * i], y = I->xy[2 * i + 1], r = I->radius[i];
        if (!std::isfinite(x) || !std::isfinite(y) || !(r > 0) || !(I->kp[i] > 0))
            return gs_fail(c, GS_ERR_ARG, "disk " + std::to_string(i) + ": bad centre, radius or kp");
        if (x < -0.5 * d || x >= 0.5 * d)
            return gs_fail(c, GS_ERR_GEOMETRY, "disk " + std::to_string(i) + ": centre outside [-d/2, d/2)");
        if (y + r >= c->h1_min || y - r <= c->h2_max)
            return gs_fail(c, GS_ERR_GEOMETRY, "disk " + std::to_string(i) + " crosses an interface band");
    }
    // minimum-image overlap test on a cell grid
    double rmax = 0;
    for (int i = 0; i < I->M; ++i) rmax = std::max(rmax, I->radius[i]);
    double cell = 2.0 * rmax;
    int ncx = std::max(1, (int)(d / cell));
    double cw = d / ncx;
    std::vector<std::vector<int>> grid;
    double ylo = c->h2_max, yhi = c->h1_min;
    int ncy = std::max(1, (int)((yhi - ylo) / cw) + 1);
    grid.resize((size_t)ncx * ncy);
    auto cx_of = [&](double x) { return std::min(ncx - 1, std::max(0, (int)((x + 0.5 * d) / cw))); };
    auto cy_of = [&](double y) { return std::min(ncy - 1, std::max(0, (int)((y - ylo) / cw))); };
    for (int i = 0; i < I->M; ++i) grid[(size_t)cy_of(I->xy[2 * i + 1]) * ncx + cx_of(I->xy[2 * i])].push_back(i);
    for (int i = 0; i < I->M; ++i) {
        int gx = cx_of(I->xy[2 * i]), gy = cy_of(I->xy[2 * i + 1]);
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                int yy = gy + oy;
                if (yy < 0 || yy >= ncy) continue;
                int xx = ((gx + ox) % ncx + ncx) % ncx;
                for (int j : grid[(size_t)yy * ncx + xx]) {
                    if (j <= i) continue;
                    double dx = std::fabs(I->xy[2 * i] - I->xy[2 * j]);
                    dx = std::min(dx, d - dx);
                    double dy = I->xy[2 * i + 1] - I->xy[2 * j + 1];
                    double rr = I->radius[i] + I->radius[j];
                    if (dx * dx + dy * dy <= rr * rr)
                        return gs_fail(c, GS_ERR_GEOMETRY,
                                       "disks " + std::to_string(i) + " and " + std::to_string(j) + " overlap");
                }
            }
    }
    // smallest centre distance (minimum image; a disk's own images are d away): for each disk,
    // rings of cells outward until the ring is farther than the best distance found
    double dmin = d;
    for (int i = 0; i < I->M; ++i) {
        const int gx = cx_of(I->xy[2 * i]), gy = cy_of(I->xy[2 * i + 1]);
        for (int ring = 0; ring <= std::max(ncx, ncy); ++ring) {
            if ((ring - 1) * cw > dmin) break;
            for (int oy = -ring; oy <= ring; ++oy) {
                const int yy = gy + oy;
                if (yy < 0 || yy >= ncy) continue;
                for (int ox = -ring; ox <= ring; ++ox) {
                    if (std::max(std::abs(ox), std::abs(oy)) != ring) continue;   // the ring only
                    const int xx = ((gx + ox) % ncx + ncx) % ncx;
                    for (int j : grid[(size_t)yy * ncx + xx]) {
                        if (j == i) continue;
                        double dx = std::fabs(I->xy[2 * i] - I->xy[2 * j]);
                        dx = std::min(dx, d - dx);
                        const double dy = I->xy[2 * i + 1] - I->xy[2 * j + 1];
                        dmin = std::min(dmin, std::sqrt(dx * dx + dy * dy));
                    }
                }
            }
        }
    }
    free_geometry(c);
    c->M = I->M;
    c->p = I->p;
    c->nc = 2 * I->p + 1;
    c->min_center_dist = dmin;
    GS_TRY(dalloc(c, &c->xy, 2 * (size_t)c->M));
    GS_TRY(dalloc(c, &c->radius, c->M));
    GS_TRY(dalloc(c, &c->kp, c->M));
    GS_TRY(dalloc(c, &c->s, (size_t)c->M * c->nc));
    GS_CUDA(c, cudaMemcpyAsync(c->xy, I->xy, sizeof(double) * 2 * c->M, cudaMemcpyHostToDevice, c->stream));
    GS_CUDA(c, cudaMemcpyAsync(c->radius, I->radius, sizeof(double) * c->M, cudaMemcpyHostToDevice, c->stream));
    GS_CUDA(c, cudaMemcpyAsync(c->kp, I->kp, sizeof(double) * c->M, cudaMemcpyHostToDevice, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    dfree(c->kp_im);   // new inclusions are lossless until gs_set_inclusion_loss
    dfree(c->star_phi);   // and disks until gs_set_inclusions_star says otherwise
    dfree(c->S0);
    dfree(c->Sblk);
    c->is_star = false;
    c->radius_h.assign(I->radius, I->radius + c->M);
    c->kp_h.assign(I->kp, I->kp + c->M);
    c->have_inc = true;
    return GS_OK;
}

int gs_set_inclusions_star(gs_ctx *c, const gs_star_inclusions *I) {
    CTX_GUARD(c);
    if (!I || I->M < 1 || !I->xy || !I->phi) return gs_fail(c, GS_ERR_ARG, "need M >= 1, xy and phi");
    if (!(I->a1 > 0.0) || !(std::fabs(I->a2) < I->a1) || I->a3 < 0 || I->a3 > 64 || !(I->kp > 0.0) ||
        I->n_nodes < 16 || I->n_nodes > 1024 || (I->n_nodes & 1))
        return gs_fail(c, GS_ERR_ARG, "star: a1 > |a2|, 0 <= a3 <= 64, kp > 0, n_nodes even in [16, 1024]");
    for (int i = 0; i < I->M; ++i)
        if (!std::isfinite(I->phi[i])) return gs_fail(c, GS_ERR_ARG, "non-finite rotation angle");
    // the enclosing disks (radius a1 + |a2|) carry the geometry checks and the multipole expansions
    std::vector<double> rad(I->M, I->a1 + std::fabs(I->a2)), kp(I->M, I->kp);
    gs_inclusions D{I->M, I->p, I->xy, rad.data(), kp.data()};
    GS_TRY(gs_set_inclusions(c, &D));
    GS_TRY(dalloc(c, &c->star_phi, c->M));
    GS_TRY(dalloc(c, &c->Sblk, (size_t)c->M * c->nc * c->nc));
    GS_CUDA(c, cudaMemcpyAsync(c->star_phi, I->phi, sizeof(double) * c->M, cudaMemcpyHostToDevice, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    c->star.a1 = I->a1;
    c->star.a2 = I->a2;
    c->star.a3 = I->a3;
    c->star.kp = I->kp;
    c->star.n_nodes = I->n_nodes;
    c->is_star = true;
    return GS_OK;
}

int gs_get_scattering_blocks(gs_ctx *c, gs_c128 *S_dev) {
    CTX_GUARD(c);
    if (!c->factored) return gs_fail(c, GS_ERR_STATE, "gs_factor has not run");
    if (!S_dev) return gs_fail(c, GS_ERR_ARG, "null output");
    const long nc = c->nc, M = c->M;
    if (c->Sblk) {
        GS_CUDA(c, cudaMemcpyAsync(S_dev, c->Sblk, sizeof(cplx) * M * nc * nc, cudaMemcpyDeviceToDevice, c->stream));
    } else {   // disks: the diagonal blocks
        std::vector<cplx> h((size_t)M * nc), out((size_t)M * nc * nc, C(0, 0));
        GS_CUDA(c, cudaMemcpyAsync(h.data(), c->s, sizeof(cplx) * M * nc, cudaMemcpyDeviceToHost, c->stream));
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
        for (long i = 0; i < M; ++i)
            for (long m = 0; m < nc; ++m) out[(i * nc + m) * nc + m] = h[i * nc + m];
        GS_CUDA(c, cudaMemcpyAsync(S_dev, out.data(), sizeof(cplx) * out.size(), cudaMemcpyHostToDevice, c->stream));
    }
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

int gs_set_polarization(gs_ctx *c, int pol) {
    CTX_GUARD(c);
    if (pol != GS_TM && pol != GS_TE) return gs_fail(c, GS_ERR_ARG, "polarisation must be GS_TM or GS_TE");
    if (pol != c->pol) {
        free_factor(c);   // the grating's matrix, right-hand side and the disk coefficients change
        c->pol = pol;
    }
    return GS_OK;
}

int gs_set_inclusion_loss(gs_ctx *c, const double *kp_im) {
    CTX_GUARD(c);
    if (!c->have_inc) return gs_fail(c, GS_ERR_STATE, "gs_set_inclusions must come first");
    free_geometry(c);
    dfree(c->kp_im);
    if (!kp_im) return GS_OK;
    bool any = false;
    for (int i = 0; i < c->M; ++i) {
        if (!std::isfinite(kp_im[i]) || kp_im[i] < 0.0)
            return gs_fail(c, GS_ERR_ARG, "disk " + std::to_string(i) + ": Im kp must be finite and >= 0");
        if (kp_im[i] > 0.0 && std::hypot(c->kp_h[i], kp_im[i]) * c->radius_h[i] > 12.0)
            return gs_fail(c, GS_ERR_ARG, "disk " + std::to_string(i) + ": |kp R| > 12 for a lossy disk");
        any = any || kp_im[i] > 0.0;
    }
    if (!any) return GS_OK;
    GS_TRY(dalloc(c, &c->kp_im, c->M));
    GS_CUDA(c, cudaMemcpyAsync(c->kp_im, kp_im, sizeof(double) * c->M, cudaMemcpyHostToDevice, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

int gs_factor(gs_ctx *c) {
    CTX_GUARD(c);
    if (!c->have_layers || !c->have_inc || c->thetas.empty())
        return gs_fail(c, GS_ERR_STATE, "set layers, incidence and inclusions before gs_factor");
    const Layout &ly = c->lay;
    GS_TRY(gs_ensure_grating(c));
    // 2. inclusion-dependent parts: S, B_phys, C, solver workspace
    free_geometry(c);
    const int n = c->n();
    GS_TRY(dalloc(c, &c->v1, n));
    GS_TRY(dalloc(c, &c->v2, n));
    GS_TRY(dalloc(c, &c->v3, n));
    GS_TRY(dalloc(c, &c->v4, n));
    GS_TRY(dalloc(c, &c->v5, n));
    GS_TRY(dalloc(c, &c->v6, n));
    c->part_elems = gs_translate_scratch_elems(c->M, c->p);
    GS_TRY(dalloc(c, &c->part, c->part_elems));
    GS_TRY(dalloc(c, &c->b32, n));
    GS_TRY(dalloc(c, &c->img32, 3 * (size_t)c->M));
    GS_TRY(dalloc(c, &c->b3pad, (size_t)((3L * c->M + 31) / 32) * 32 * c->nc));
    GS_TRY(dalloc(c, &c->xdf, n));
    GS_TRY(dalloc(c, &c->iflag, 1));
    GS_TRY(gs_build_images_c64(c, c->xy, c->M, c->img32, c->stream));
    c->kdim = 200;
    GS_TRY(dalloc(c, &c->Vk, (size_t)(c->kdim + 1) * n));
    GS_TRY(dalloc(c, &c->kv1, n));
    GS_TRY(dalloc(c, &c->kv2, n));
    GS_TRY(dalloc(c, &c->Hh, (size_t)(c->kdim + 1) * c->kdim));
    GS_TRY(dalloc(c, &c->cs, c->kdim + 1));
    GS_TRY(dalloc(c, &c->sn, c->kdim + 1));
    GS_TRY(dalloc(c, &c->gg, c->kdim + 1));
    GS_TRY(dalloc(c, &c->yy, c->kdim + 1));
    GS_TRY(gs_mie(c));
    if (c->is_star) GS_TRY(gs_star_blocks(c));
    {
        // translation coefficient table for the FP64 product, when it fits the memory budget
        size_t bytes = sizeof(cplx) * gs_pair_table_elems(c->M, c->p);
        size_t fr = 0, totm = 0;
        GS_CUDA(c, cudaMemGetInfo(&fr, &totm));
        double budget = c->table_budget_gb >= 0 ? c->table_budget_gb * 1e9 : 0.5 * (double)fr;
        if ((double)bytes <= budget) {
            if (cudaMalloc((void **)&c->htab, bytes) == cudaSuccess) {
                GS_TRY(gs_build_pair_table(c));
            } else {
                cudaGetLastError();
                c->htab = nullptr;
            }
        }
    }
    for (auto &a : c->ang) {
        GS_TRY(dalloc(c, &a.B, (size_t)n * ly.nB()));
        GS_TRY(dalloc(c, &a.Cm, (size_t)ly.nC() * n));
        GS_TRY(dalloc(c, &a.beta, n));
        GS_CUDA(c, cudaMemsetAsync(a.beta, 0, sizeof(cplx) * n, c->stream));
        GS_TRY(gs_assemble_B(c, a, a.B));
        GS_TRY(gs_assemble_C(c, a, a.Cm));
    }
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    c->factored = true;
    return GS_OK;
}

int gs_dims(gs_ctx *c, int *rows, int *cols, int *n, int *nB, int *nC) {
    if (!c) return GS_ERR_ARG;
    if (!c->have_layers) return gs_fail(c, GS_ERR_STATE, "no layers");
    if (rows) *rows = c->lay.rows;
    if (cols) *cols = c->lay.cols;
    if (n) *n = c->have_inc ? c->n() : 0;
    if (nB) *nB = c->lay.nB();
    if (nC) *nC = c->lay.nC();
    return GS_OK;
}

int gs_get_A(gs_ctx *c, int angle, gs_c128 *A_dev) {
    CTX_GUARD(c);
    GS_TRY(check_angle(c, angle));
    if (!A_dev) return gs_fail(c, GS_ERR_ARG, "null output");
    GS_TRY(gs_assemble_A(c, c->ang[angle], (cplx *)A_dev, c->lay.rows));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

int gs_get_f(gs_ctx *c, int angle, gs_c128 *f_dev) {
    CTX_GUARD(c);
    GS_TRY(check_angle(c, angle));
    if (!f_dev) return gs_fail(c, GS_ERR_ARG, "null output");
    GS_CUDA(c, cudaMemcpyAsync(f_dev, c->ang[angle].f, sizeof(cplx) * c->lay.rows, cudaMemcpyDeviceToDevice,
                               c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

int gs_get_coupling(gs_ctx *c, int angle, gs_c128 *B_dev, gs_c128 *C_dev) {
    CTX_GUARD(c);
    GS_TRY(check_angle(c, angle));
    const AngleData &a = c->ang[angle];
    size_t n = c->n();
    if (B_dev)
        GS_CUDA(c, cudaMemcpyAsync(B_dev, a.B, sizeof(cplx) * n * c->lay.nB(), cudaMemcpyDeviceToDevice, c->stream));
    if (C_dev)
        GS_CUDA(c, cudaMemcpyAsync(C_dev, a.Cm, sizeof(cplx) * n * c->lay.nC(), cudaMemcpyDeviceToDevice, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

int gs_get_scattering(gs_ctx *c, gs_c128 *s_dev) {
    CTX_GUARD(c);
    if (!c->factored) return gs_fail(c, GS_ERR_STATE, "gs_factor has not run");
    if (!s_dev) return gs_fail(c, GS_ERR_ARG, "null output");
    GS_CUDA(c, cudaMemcpyAsync(s_dev, c->s, sizeof(cplx) * c->n(), cudaMemcpyDeviceToDevice, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

int gs_pinv_apply(gs_ctx *c, int angle, const gs_c128 *g_dev, gs_c128 *x_dev) {
    CTX_GUARD(c);
    GS_TRY(check_angle(c, angle));
    if (!g_dev || !x_dev) return gs_fail(c, GS_ERR_ARG, "null vector");
    GS_TRY(gs_pinv_impl(c, c->ang[angle], (const cplx *)g_dev, (cplx *)x_dev));
    return GS_OK;
}

int gs_translate(gs_ctx *c, int angle, const gs_c128 *beta_dev, gs_c128 *alpha_dev, int precision) {
    CTX_GUARD(c);
    GS_TRY(check_angle(c, angle));
    if (!beta_dev || !alpha_dev || beta_dev == (const gs_c128 *)alpha_dev)
        return gs_fail(c, GS_ERR_ARG, "null or aliased vectors");
    if (precision != GS_FP64 && precision != GS_C64) return gs_fail(c, GS_ERR_ARG, "bad precision");
    GS_TRY(gs_translate_impl(c, c->ang[angle], (const cplx *)beta_dev, (cplx *)alpha_dev, precision));
    return precision == GS_C64 && c->tab32.h ? gs_check_table_wait(c) : GS_OK;
}

int gs_apply(gs_ctx *c, int angle, const gs_c128 *x_dev, gs_c128 *y_dev, int precision) {
    CTX_GUARD(c);
    GS_TRY(check_angle(c, angle));
    if (!x_dev || !y_dev || x_dev == (const gs_c128 *)y_dev) return gs_fail(c, GS_ERR_ARG, "null or aliased vectors");
    if (precision != GS_FP64 && precision != GS_C64) return gs_fail(c, GS_ERR_ARG, "bad precision");
    GS_TRY(gs_apply_impl(c, c->ang[angle], (const cplx *)x_dev, (cplx *)y_dev, precision));
    return precision == GS_C64 && c->tab32.h ? gs_check_table_wait(c) : GS_OK;
}

int gs_rhs(gs_ctx *c, int angle, gs_c128 *b_dev) {
    CTX_GUARD(c);
    GS_TRY(check_angle(c, angle));
    if (!b_dev) return gs_fail(c, GS_ERR_ARG, "null output");
    return gs_rhs_impl(c, c->ang[angle], (cplx *)b_dev);
}

int gs_solve(gs_ctx *c, int angle, const gs_solve_opts *o, const gs_c128 *beta0_dev) {
    CTX_GUARD(c);
    GS_TRY(check_angle(c, angle));
    if (!o || !(o->tol > 0) || o->maxit < 1 || o->restart < 1)
        return gs_fail(c, GS_ERR_ARG, "tol > 0, maxit >= 1, restart >= 1 required");
    if (o->precision != GS_FP64 && o->precision != GS_C64) return gs_fail(c, GS_ERR_ARG, "bad precision");
    return gs_solve_impl(c, c->ang[angle], *o, (const cplx *)beta0_dev);
}

int gs_get_beta(gs_ctx *c, int angle, gs_c128 *beta_dev) {
    CTX_GUARD(c);
    GS_TRY(check_angle(c, angle));
    if (!beta_dev) return gs_fail(c, GS_ERR_ARG, "null output");
    GS_CUDA(c, cudaMemcpyAsync(beta_dev, c->ang[angle].beta, sizeof(cplx) * c->n(), cudaMemcpyDeviceToDevice,
                               c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    return GS_OK;
}

int gs_stats(gs_ctx *c, int angle, int *iters, double *relres) {
    if (!c) return GS_ERR_ARG;
    GS_TRY(check_angle(c, angle));
    if (iters) *iters = c->ang[angle].iters;
    if (relres) *relres = c->ang[angle].relres;
    return GS_OK;
}

int gs_stats_refinement(gs_ctx *c, int angle, int *outer) {
    if (!c || !outer) return GS_ERR_ARG;
    GS_TRY(check_angle(c, angle));
    *outer = c->ang[angle].outer;
    return GS_OK;
}

int gs_bragg(gs_ctx *c, int angle, int *n_top, int *orders_top, gs_c128 *cc, int *n_bot, int *orders_bot,
             gs_c128 *dd, double *flux_err) {
    CTX_GUARD(c);
    GS_TRY(check_angle(c, angle));
    if (!n_top || !orders_top || !cc || !n_bot || !orders_bot || !dd || !flux_err)
        return gs_fail(c, GS_ERR_ARG, "null output");
    const AngleData &a = c->ang[angle];
    const int K = c->lay.K, K2 = 2 * K + 1;
    std::vector<cplx> cd(2 * K2);
    double flux = 0;
    GS_TRY(gs_bragg_impl(c, a, cd.data(), &flux));
    std::vector<cplx> k1n(K2), k3n(K2);
    GS_CUDA(c, cudaMemcpy(k1n.data(), a.k1n, sizeof(cplx) * K2, cudaMemcpyDeviceToHost));
    GS_CUDA(c, cudaMemcpy(k3n.data(), a.k3n, sizeof(cplx) * K2, cudaMemcpyDeviceToHost));
    int nt = 0, nbt = 0;
    bool finite = std::isfinite(flux);
    for (int q = 0; q < K2; ++q) {
        if (k1n[q].y == 0.0 && k1n[q].x > 0.0) {
            orders_top[nt] = q - K;
            cc[nt].re = cd[q].x;
            cc[nt].im = cd[q].y;
            finite = finite && std::isfinite(cd[q].x) && std::isfinite(cd[q].y);
            ++nt;
        }
        if (k3n[q].y == 0.0 && k3n[q].x > 0.0) {
            orders_bot[nbt] = q - K;
            dd[nbt].re = cd[K2 + q].x;
            dd[nbt].im = cd[K2 + q].y;
            finite = finite && std::isfinite(cd[K2 + q].x) && std::isfinite(cd[K2 + q].y);
            ++nbt;
        }
    }
    *n_top = nt;
    *n_bot = nbt;
    *flux_err = flux;
    return finite ? GS_OK : gs_fail(c, GS_ERR_NUMERIC, "non-finite Bragg amplitude");
}

int gs_set_table_budget(gs_ctx *c, double budget_gb) {
    if (!c) return GS_ERR_ARG;
    c->table_budget_gb = budget_gb;
    return GS_OK;
}

int gs_launch_count(gs_ctx *c, unsigned long long *count) {
    if (!c || !count) return GS_ERR_ARG;
    *count = c->nlaunch;
    return GS_OK;
}

int gs_profile(gs_ctx *c, int enable) {
    CTX_GUARD(c);
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    c->prof_on = enable != 0;
    c->prof_used = 0;
    return GS_OK;
}

int gs_profile_read(gs_ctx *c, int precision, int *launches, double *total_ms) {
    CTX_GUARD(c);
    if (!launches || !total_ms) return gs_fail(c, GS_ERR_ARG, "null output");
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    double tot = 0.0;
    int cnt = 0;
    for (size_t q = 0; q + 1 < c->prof_used; q += 2) {
        if (c->prof_prec[q / 2] != precision) continue;
        float ms = 0.f;
        GS_CUDA(c, cudaEventElapsedTime(&ms, c->prof_ev[q], c->prof_ev[q + 1]));
        tot += ms;
        ++cnt;
    }
    *launches = cnt;
    *total_ms = tot;
    return GS_OK;
}

}  // extern "C"
