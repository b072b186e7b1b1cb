// Lockstep solves of one inclusion geometry at many incidence angles (Sec. 2 Eqs. quasi, rad1-rad2:
// each angle is its own quasi-periodic problem, with Bloch phase a_r = exp(i k1 cos(theta_r) d)).
//
//  * Translation: the R angles' coefficient vectors go through one tensor-core product per operator
//    part (tcgen05, gs_tc.cu): the geometry's operator [T_-1 T_0 T_1] and the coefficients are each
//    split into three bfloat16 parts (~24 significant bits together, the precision of FP32) and the
//    six products of parts whose orders add up to at most 2 are accumulated in FP32 -- the accuracy
//    of the complex64 translation -- for all R angles at the cost of streaming the operator three
//    times.
//  * Low rank: per angle, since the grating factorisation, B_phys and C depend on the angle: C x in
//    double-float arithmetic, U^* and V Sigma in double-float, complex64 B_phys, fused combination
//    (gs_lowrank_c64).
//  * GMRES: segmented Arnoldi steps over the R angles (gs_seg.cuh, the kernels of the batched
//    solver), each step captured once as a CUDA graph and replayed; the host reads one residual
//    estimate per angle per step and masks converged angles.
//  * Refinement: FP64 residual of every open angle (the table-driven FP64 translation), inner
//    solves of the corrections on the operator above to max(inner_tol, tol / (2 rel)) per angle.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gs_internal.h"
#include "gs_seg.cuh"

struct gs_angles {
    int R = 0, kdim = 0;
    long n = 0, N = 0;                 // unknowns per angle, R n
    cudaStream_t st = nullptr;         // own (capturable) stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    Geo *geo = nullptr;                // R segments of M targets
    int *gid = nullptr;                // segment of each of the R M targets
    cplx *alpha = nullptr;             // R image phases
    cplx *X = nullptr, *Y = nullptr, *T = nullptr, *b = nullptr, *r = nullptr, *dx = nullptr, *x = nullptr;
    int *active = nullptr, *jdev = nullptr, *kk = nullptr, *err = nullptr;
    cplx *Vk = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *gg = nullptr, *yy = nullptr, *hp = nullptr;
    double *nrm = nullptr, *res = nullptr, *npart = nullptr;   // R, R, R x SEG_NQ
    float2 *w32 = nullptr, *cf32 = nullptr;                      // N, R x (kdim+1): complex64 CGS2 operands
    double *hbuf = nullptr;            // pinned host: R residuals + the error flag
    int mode = 0;                      // inner translation: 0 tensor-core product of all R angles,
                                       // 1 complex64 table, one launch per angle
    cudaGraphExec_t step[2] = {nullptr, nullptr};   // step graph per mode
    unsigned long long step_kernels[2] = {0, 0};    // kernels in one replay of each step graph
    const void *key[2][4] = {};                     // operator and scratch buffers each graph uses
};

namespace {

inline int nblk(long n, int t = 256) { return (int)((n + t - 1) / t); }

template <typename T>
int aalloc(gs_ctx *c, T **p, size_t n) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * std::max<size_t>(n, 1));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return gs_fail(c, GS_ERR_OOM, std::string("cudaMalloc (multi-angle solve): ") + cudaGetErrorString(e));
    }
    return GS_OK;
}
template <typename T>
void afree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void angles_free(gs_angles *A) {
    if (!A) return;
    afree(A->geo);
    afree(A->gid);
    afree(A->alpha);
    afree(A->X);
    afree(A->Y);
    afree(A->T);
    afree(A->b);
    afree(A->r);
    afree(A->dx);
    afree(A->x);
    afree(A->active);
    afree(A->jdev);
    afree(A->kk);
    afree(A->err);
    afree(A->Vk);
    afree(A->H);
    afree(A->cs);
    afree(A->sn);
    afree(A->gg);
    afree(A->yy);
    afree(A->hp);
    afree(A->npart);
    afree(A->w32);
    afree(A->cf32);
    afree(A->nrm);
    afree(A->res);
    if (A->hbuf) cudaFreeHost(A->hbuf);
    for (int q = 0; q < 2; ++q)
        if (A->step[q]) cudaGraphExecDestroy(A->step[q]);
    if (A->st) cudaStreamDestroy(A->st);
    if (A->ev_in) cudaEventDestroy(A->ev_in);
    if (A->ev_out) cudaEventDestroy(A->ev_out);
    delete A;
}

// workspace for R angles of the current geometry and a Krylov dimension of up to 512
int angles_setup(gs_ctx *c, int restart) {
    const int R = (int)c->ang.size();
    const long n = c->n();
    const int kdim = std::max(1, std::min(restart, 512));
    gs_angles *A = c->angles;
    if (A && A->R == R && A->n == n && A->kdim >= kdim) return GS_OK;
    gs_angles_destroy(c);
    A = new gs_angles();
    c->angles = A;
    A->R = R;
    A->n = n;
    A->N = (long)R * n;
    A->kdim = kdim;
    GS_CUDA(c, cudaStreamCreateWithFlags(&A->st, cudaStreamNonBlocking));
    GS_CUDA(c, cudaEventCreateWithFlags(&A->ev_in, cudaEventDisableTiming));
    GS_CUDA(c, cudaEventCreateWithFlags(&A->ev_out, cudaEventDisableTiming));
    std::vector<Geo> geo(R);
    std::vector<int> gid((size_t)R * c->M);
    std::vector<cplx> al(R);
    for (int r = 0; r < R; ++r) {
        geo[r] = Geo{c->M, 0, (int)(r * n)};
        for (int i = 0; i < c->M; ++i) gid[(size_t)r * c->M + i] = r;
        al[r] = c->ang[r].alpha;
    }
    const long N = A->N;
    const int ld = kdim + 1;
    GS_TRY(aalloc(c, &A->geo, R));
    GS_TRY(aalloc(c, &A->gid, gid.size()));
    GS_TRY(aalloc(c, &A->alpha, R));
    GS_CUDA(c, cudaMemcpy(A->geo, geo.data(), sizeof(Geo) * R, cudaMemcpyHostToDevice));
    GS_CUDA(c, cudaMemcpy(A->gid, gid.data(), sizeof(int) * gid.size(), cudaMemcpyHostToDevice));
    GS_CUDA(c, cudaMemcpy(A->alpha, al.data(), sizeof(cplx) * R, cudaMemcpyHostToDevice));
    for (cplx **v : {&A->X, &A->Y, &A->T, &A->b, &A->r, &A->dx, &A->x}) GS_TRY(aalloc(c, v, N));
    GS_TRY(aalloc(c, &A->active, R));
    GS_TRY(aalloc(c, &A->jdev, 1));
    GS_TRY(aalloc(c, &A->kk, R));
    GS_TRY(aalloc(c, &A->err, 1));
    // complex64 Krylov basis (the inner solves), held in a complex128-typed buffer of half the size
    GS_TRY(aalloc(c, &A->Vk, ((size_t)ld * N + 1) / 2));
    GS_TRY(aalloc(c, &A->H, (size_t)R * kdim * ld));
    for (cplx **v : {&A->cs, &A->sn, &A->gg, &A->yy, &A->hp}) GS_TRY(aalloc(c, v, (size_t)R * ld));
    GS_TRY(aalloc(c, &A->cf32, (size_t)R * ld));
    GS_TRY(aalloc(c, &A->w32, (size_t)A->N));
    GS_TRY(aalloc(c, &A->npart, (size_t)R * SEG_NQ));
    GS_TRY(aalloc(c, &A->nrm, R));
    GS_TRY(aalloc(c, &A->res, R));
    GS_CUDA(c, cudaMallocHost((void **)&A->hbuf, sizeof(double) * (R + 1)));
    GS_CUDA(c, cudaMemset(A->err, 0, sizeof(int)));
    return GS_OK;
}

// y_r = x_r - s T(a_r) x_r + s B_phys,r A_r^+ C_r x_r for every angle r (the mixed inner operator)
// inner operator of every angle; act (nullable): device flags of the angles whose translation is needed
// (mode 1 skips the others; the tensor-core product always forms all R)
int angles_apply_c64(gs_ctx *c, gs_angles *A, const cplx *x, cplx *y, const int *act) {
    if (A->mode == 1) {
        for (int r = 0; r < A->R; ++r)
            GS_TRY(gs_tab32_translate(c, c->tab32, c->M, c->p, x + (size_t)r * A->n, c->ang[r].alpha, c->b3pad,
                                      c->part, c->part_elems, A->T + (size_t)r * A->n, act ? act + r : nullptr,
                                      c->stream));
    } else {
        GS_TRY(gs_tc_split_translate(c, A->R, A->alpha, x, A->T, A->err, c->stream));
    }
    for (int r = 0; r < A->R; ++r)
        GS_TRY(gs_lowrank_c64(c, c->ang[r], x + (size_t)r * A->n, A->T + (size_t)r * A->n, y + (size_t)r * A->n));
    return GS_OK;
}

int angles_norms(gs_ctx *c, gs_angles *A, const cplx *v, std::vector<double> &out) {
    GS_COUNT_LAUNCH(c);
    k_seg_norm<<<A->R, 256, 0, c->stream>>>(v, A->geo, c->nc, nullptr, A->nrm, nullptr, 0, 0, nullptr);
    GS_CHECK_LAUNCH(c);
    GS_CUDA(c, cudaMemcpyAsync(A->hbuf, A->nrm, sizeof(double) * A->R, cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    out.assign(A->hbuf, A->hbuf + A->R);
    return GS_OK;
}

// one Arnoldi step (complex64 basis) for every active angle, j read from A->jdev
int angles_step(gs_ctx *c, gs_angles *A) {
    cudaStream_t st = c->stream;
    const long N = A->N;
    const int ld = A->kdim + 1, eb = nblk(N), R = A->R, nc = c->nc;
    float2 *V = (float2 *)A->Vk;
    GS_COUNT_LAUNCH(c);
    k_seg_fetch<float2><<<eb, 256, 0, st>>>(V, N, A->jdev, A->X);
    GS_TRY(angles_apply_c64(c, A, A->X, A->Y, A->active));
    const SegStep ss{A->geo, A->gid, A->active, A->jdev, A->H, A->hp, A->cs, A->sn, A->gg, A->nrm, A->res, A->npart,
                     A->w32, A->cf32, N, R, A->kdim, nc};
    GS_TRY(seg_cgs2<float2>(c, ss, V, A->Y, st));
    GS_COUNT_LAUNCH(c);
    k_inc<<<1, 32, 0, st>>>(A->jdev);
    GS_CHECK_LAUNCH(c);
    return GS_OK;
}

int angles_step_graph(gs_ctx *c, gs_angles *A) {
    const int q = A->mode;
    const void *key[4] = {c->tcA, c->tcA_sp[0], c->tcA_sp[1], c->sp_scratch};
    if (q == 1) {   // the complex64 table, its tiles and the translation scratch
        key[0] = c->tab32.h;
        key[1] = c->b3pad;
        key[2] = c->part;
        key[3] = nullptr;
    }
    if (A->step[q] && std::equal(key, key + 4, A->key[q])) return GS_OK;
    if (A->step[q]) {   // the buffers were rebuilt since the capture
        cudaGraphExecDestroy(A->step[q]);
        A->step[q] = nullptr;
    }
    std::copy(key, key + 4, A->key[q]);
    cudaGraph_t gph;
    const unsigned long long l0 = c->nlaunch;
    GS_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const int st = angles_step(c, A);
    cudaError_t e = cudaStreamEndCapture(c->stream, &gph);
    if (st != GS_OK) return st;
    if (e != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&A->step[q], gph, 0);
    cudaGraphDestroy(gph);
    if (e != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    A->step_kernels[q] = c->nlaunch - l0;
    c->nlaunch = l0;   // counted per replay
    return GS_OK;
}

int check_err(gs_ctx *c, gs_angles *A) {
    int herr = 0;
    GS_CUDA(c, cudaMemcpyAsync(&herr, A->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    if (herr) return gs_fail(c, GS_ERR_TIMEOUT, "tensor-core product: a device wait gave up");
    return GS_OK;
}

// lockstep restarted GMRES on the inner operator: solves L32_r x_r = rhs_r from zero until
// ||rhs_r - L32_r x_r|| <= tolabs[r] for every angle not done
int angles_gmres(gs_ctx *c, gs_angles *A, const cplx *rhs, cplx *x, const std::vector<double> &tolabs,
                 std::vector<int> &done, const std::vector<int> &cap, int restart, std::vector<int> &iters) {
    cudaStream_t st = c->stream;
    const long N = A->N;
    const int R = A->R, ld = A->kdim + 1, eb = nblk(N), nc = c->nc;
    const int kd = std::min(restart, A->kdim);
    GS_CUDA(c, cudaMemsetAsync(x, 0, sizeof(cplx) * N, st));
    std::vector<int> act(R), kk(R), used(R, 0), est_conv(R, 0);
    std::vector<double> nr;
    bool first = true;
    for (;;) {
        if (first) {
            GS_CUDA(c, cudaMemcpyAsync(A->r, rhs, sizeof(cplx) * N, cudaMemcpyDeviceToDevice, st));
        } else {
            GS_TRY(angles_apply_c64(c, A, x, A->r, nullptr));
            GS_COUNT_LAUNCH(c);
            k_vsub<<<eb, 256, 0, st>>>(rhs, A->r, N, A->r);
        }
        first = false;
        GS_TRY(angles_norms(c, A, A->r, nr));
        int nact = 0;
        for (int q = 0; q < R; ++q) {
            const double lim = est_conv[q] ? 10.0 * tolabs[q] : tolabs[q];
            act[q] = (!done[q] && nr[q] > lim && used[q] < cap[q]) ? 1 : 0;
            if (!act[q]) done[q] = 1;
            nact += act[q];
        }
        if (nact == 0) break;
        GS_CUDA(c, cudaMemcpyAsync(A->active, act.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
        GS_CUDA(c, cudaMemcpyAsync(A->nrm, nr.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
        GS_COUNT_LAUNCH(c);
        k_seg_start<float2><<<eb, 256, 0, st>>>(A->r, (float2 *)A->Vk, N, A->gid, nc, A->nrm, A->active);
        GS_COUNT_LAUNCH(c);
        k_seg_g0<<<nblk((long)R * ld), 256, 0, st>>>(A->gg, ld, A->nrm, R);
        GS_CUDA(c, cudaMemsetAsync(A->H, 0, sizeof(cplx) * (size_t)R * A->kdim * ld, st));
        GS_CUDA(c, cudaMemsetAsync(A->jdev, 0, sizeof(int), st));
        GS_TRY(angles_step_graph(c, A));
        std::fill(kk.begin(), kk.end(), 0);
        std::vector<int> live = act;
        for (int j = 0; j < kd; ++j) {
            GS_CUDA(c, cudaGraphLaunch(A->step[A->mode], st));
            c->nlaunch += A->step_kernels[A->mode];
            GS_CUDA(c, cudaMemcpyAsync(A->hbuf, A->res, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
            GS_CUDA(c, cudaStreamSynchronize(st));
            int nlive = 0;
            bool changed = false;
            for (int q = 0; q < R; ++q) {
                if (!live[q]) continue;
                iters[q] += 1;
                used[q] += 1;
                kk[q] = j + 1;
                if (A->hbuf[q] <= tolabs[q] || used[q] >= cap[q]) {
                    est_conv[q] = A->hbuf[q] <= tolabs[q];
                    live[q] = 0;
                    changed = true;
                } else {
                    ++nlive;
                }
            }
            if (nlive == 0) break;
            if (changed) GS_CUDA(c, cudaMemcpyAsync(A->active, live.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
        }
        for (int q = 0; q < R; ++q)
            if (live[q]) est_conv[q] = 0;
        GS_TRY(check_err(c, A));
        GS_CUDA(c, cudaMemcpyAsync(A->kk, kk.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
        GS_COUNT_LAUNCH(c);
        k_seg_backsolve<<<R, 256, 0, st>>>(A->H, ld, A->kdim, A->kk, A->gg, A->yy, R);
        GS_COUNT_LAUNCH(c);
        k_seg_update<float2><<<eb, 256, 0, st>>>(x, (const float2 *)A->Vk, N, A->gid, nc, A->kk, A->yy, ld);
        GS_CHECK_LAUNCH(c);
    }
    return GS_OK;
}

// the multi-angle work runs on the solver's own stream, ordered after the context stream's earlier
// work and before its later work (the context stream may be the legacy default stream, which cannot
// be captured into a graph)
struct OnAnglesStream {
    gs_ctx *c;
    cudaStream_t saved;
    explicit OnAnglesStream(gs_ctx *cc) : c(cc), saved(cc->stream) {
        gs_angles *A = c->angles;
        cudaEventRecord(A->ev_in, saved);
        cudaStreamWaitEvent(A->st, A->ev_in, 0);
        c->stream = A->st;
    }
    ~OnAnglesStream() {
        gs_angles *A = c->angles;
        cudaEventRecord(A->ev_out, A->st);
        cudaStreamWaitEvent(saved, A->ev_out, 0);
        c->stream = saved;
    }
};

}  // namespace

void gs_angles_destroy(gs_ctx *c) {
    if (c && c->angles) {
        angles_free(c->angles);
        c->angles = nullptr;
    }
}

extern "C" int gs_solve_angles(gs_ctx *c, const gs_solve_opts *o) {
    if (!c) return GS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return gs_fail(c, GS_ERR_CUDA, "cudaSetDevice");
    if (!c->factored) return gs_fail(c, GS_ERR_STATE, "gs_factor has not run");
    if (!o || !(o->tol > 0) || o->maxit < 1 || o->restart < 1) return gs_fail(c, GS_ERR_ARG, "bad options");
    if (o->precision != GS_C64 && o->precision != GS_MIXED_BF16)
        return gs_fail(c, GS_ERR_ARG, "the multi-angle solve is a mixed form (GS_C64 or GS_MIXED_BF16)");
    const int R = (int)c->ang.size();
    if (R < 1 || R > 256) return gs_fail(c, GS_ERR_ARG, "the multi-angle solve takes 1..256 angles");
    GS_TRY(angles_setup(c, o->restart));
    gs_angles *A = c->angles;
    const long n = A->n, N = A->N;
    // everything that allocates, before the step graph is captured
    for (int r = 0; r < R; ++r) GS_TRY(gs_prepare_c64(c, c->ang[r]));
    A->mode = 0;
    if (o->precision == GS_C64) {
        GS_TRY(gs_c64_range(c));
        GS_TRY(gs_ensure_table32(c));
        if (!c->tab32.h) return gs_fail(c, GS_ERR_OOM, "no room for the complex64 pair table (use GS_MIXED_BF16)");
        A->mode = 1;
    } else {
        GS_TRY(gs_tc_split_prepare(c, R));
    }
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    OnAnglesStream on(c);
    cudaStream_t st = c->stream;
    GS_CUDA(c, cudaMemsetAsync(A->err, 0, sizeof(int), st));
    // right-hand sides and their norms
    for (int r = 0; r < R; ++r) GS_TRY(gs_rhs_impl(c, c->ang[r], A->b + (size_t)r * n));
    std::vector<double> bn, rn;
    GS_TRY(angles_norms(c, A, A->b, bn));
    std::vector<double> tolabs(R);
    for (int r = 0; r < R; ++r) tolabs[r] = o->tol * bn[r];
    std::vector<int> iters(R, 0), outer(R, 0);
    const double floor_tol = o->inner_tol > 0 ? o->inner_tol : 1e-6;
    const int max_sweeps = o->max_sweeps > 0 ? o->max_sweeps : 30;
    GS_CUDA(c, cudaMemsetAsync(A->x, 0, sizeof(cplx) * N, st));
    std::vector<int> closed(R, 0);
    for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
        // FP64 residual of every open angle (closed angles keep theirs)
        if (sweep == 0) {
            GS_CUDA(c, cudaMemcpyAsync(A->r, A->b, sizeof(cplx) * N, cudaMemcpyDeviceToDevice, st));
            rn = bn;
        } else {
            for (int r = 0; r < R; ++r) {
                if (closed[r]) continue;
                cplx *xr = A->x + (size_t)r * n, *rr = A->r + (size_t)r * n;
                GS_TRY(gs_apply_impl(c, c->ang[r], xr, rr, GS_FP64));
                GS_COUNT_LAUNCH(c);
                k_vsub<<<nblk(n), 256, 0, st>>>(A->b + (size_t)r * n, rr, n, rr);
            }
            GS_CHECK_LAUNCH(c);
            std::vector<double> tmp;
            GS_TRY(angles_norms(c, A, A->r, tmp));
            for (int r = 0; r < R; ++r)
                if (!closed[r]) rn[r] = tmp[r];
        }
        std::vector<int> idone(R, 0), cap(R, 0);
        std::vector<double> itol(R, 0.0);
        int open = 0;
        for (int r = 0; r < R; ++r) {
            if (!closed[r]) outer[r] = sweep;
            if (closed[r] || rn[r] <= tolabs[r] || bn[r] == 0.0 || iters[r] >= o->maxit) {
                closed[r] = 1;
                idone[r] = 1;
                continue;
            }
            ++open;
            const double rel = rn[r] / bn[r];
            itol[r] = std::max(floor_tol, 0.5 * o->tol / rel) * rn[r];
            cap[r] = o->maxit - iters[r];
        }
        if (open == 0 || sweep == max_sweeps) break;
        GS_TRY(angles_gmres(c, A, A->r, A->dx, itol, idone, cap, o->restart, iters));
        // x += dx on the open angles (dx is zero on the others: their segments were never active)
        for (int r = 0; r < R; ++r) {
            if (closed[r]) continue;
            GS_COUNT_LAUNCH(c);
            k_vadd<<<nblk(n), 256, 0, st>>>(A->x + (size_t)r * n, A->dx + (size_t)r * n, n);
        }
        GS_CHECK_LAUNCH(c);
    }
    if (A->mode == 1) GS_TRY(gs_check_table_wait(c));
    bool ok = true;
    for (int r = 0; r < R; ++r) {
        AngleData &a = c->ang[r];
        GS_CUDA(c, cudaMemcpyAsync(a.beta, A->x + (size_t)r * n, sizeof(cplx) * n, cudaMemcpyDeviceToDevice, st));
        a.iters = iters[r];
        a.outer = outer[r];
        a.relres = bn[r] > 0.0 ? rn[r] / bn[r] : 0.0;
        if (a.relres > o->tol) ok = false;
    }
    GS_CUDA(c, cudaStreamSynchronize(st));
    return ok ? GS_OK : GS_ERR_NOT_CONVERGED;
}
