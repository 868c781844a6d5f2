// rf_api.cu -- host driver behind the C ABI of include/rf.h.
//
// Owns the device memory of a context, the EBATS controller (Sec. 2.2), the
// Picard loop with its global max|dh| exit test (Sec. 2.3) and the water
// balance bookkeeping.  Every step of the numerical path runs in the CUDA
// kernels of closure_assemble.cu and pcg.cu; the host only sequences them and
// reads back a few scalars per Picard iteration.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dic.cuh"
#include "mg.cuh"
#include "nn.cuh"
#include "rf.h"
#include "rf_internal.cuh"

using namespace rf;

namespace {

thread_local std::string g_err;

rf_status fail(rf_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

#define CUDA_TRY(x)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (x);                                                                \
        if (e_ != cudaSuccess) return fail(RF_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct BcSeries {
    int type = BC_ZERO_FLUX;
    std::vector<double> t, v;
};

// simulated-time comparison tolerance
double t_tol(double t) { return 1e-9 * (std::fabs(t) > 1.0 ? std::fabs(t) : 1.0); }

}  // namespace

void rf::set_last_error(const char *msg) { g_err = msg; }

struct rf_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    rf_allocator alloc{};
    bool has_alloc = false;
    std::vector<void *> allocations;

    Grid g{};
    int nblk = 1;
    int n_active = 0;
    rf_solver_params prm{};
    std::vector<uint8_t> flags_h;
    BcSeries bc[6];

    // device arrays (N elements unless noted)
    uint8_t *flags = nullptr, *zone = nullptr;
    double *Ks = nullptr;
    DevSoil *soils = nullptr;   // 256 entries
    FFTables *fftab = nullptr;
    double *h = nullptr, *hk = nullptr, *x = nullptr, *theta_n = nullptr, *theta_k = nullptr;
    double *K[2] = {nullptr, nullptr}, *Can = nullptr, *c = nullptr, *b = nullptr;
    double *s0 = nullptr;                // modified Picard: storage part of b (water balance)
    double *Tx = nullptr, *Ty = nullptr, *Tz = nullptr, *diag = nullptr, *dinv = nullptr;
    double *r = nullptr, *z = nullptr, *p[2] = {nullptr, nullptr}, *q = nullptr;
    float *K32 = nullptr, *cb32 = nullptr, *dinv32 = nullptr, *r32 = nullptr, *z32 = nullptr;
    float *p32[2] = {nullptr, nullptr}, *q32 = nullptr, *d32 = nullptr;
    double *partials = nullptr;
    unsigned int *ticket = nullptr;
    CgScal *sc = nullptr, *sc_in = nullptr;
    StepResults *res = nullptr;
    StepParams *sp = nullptr;
    PicardCtl *ctl = nullptr;
    unsigned long long *ctr = nullptr;
    // pinned host mirrors
    CgScal *sc_h = nullptr, *sc_in_h = nullptr;
    StepResults *res_h = nullptr;
    StepParams *sp_h = nullptr;
    PicardCtl *ctl_h = nullptr;
    unsigned long long *ctr_h = nullptr;

    TmaMaps32 tma{};                     // tensor maps of the FP32 inner-solve arrays
    bool tma_ok = false;
    int *dev_fault = nullptr, *fault_h = nullptr;   // set by a device wait that ran out

    MgHierarchy mg;                      // multigrid levels (RF_PRECOND_MG)
    float *dic_diag = nullptr, *dic_rd = nullptr;   // DIC diagonal and pivots (RF_PRECOND_DIC)
    bool mg_alloc = false;

    // CUDA graphs: a whole Picard attempt, and a stand-alone linear solve
    cudaStream_t cap = nullptr;          // private capture stream
    cudaGraph_t picard_graph = nullptr, solve_graph = nullptr;
    cudaGraphExec_t picard_exec = nullptr, solve_exec = nullptr;

    // learned warm start: each step's first attempt starts from the network's guess
    rf_nn *ws_net = nullptr;
    nn::WsScales ws_sc{};
    long long ws_guesses = 0, ws_fallbacks = 0;

    // BDF2: theta*(h^{n-1}) and the previous step size (0: no history)
    double *theta_p = nullptr;
    double dt_prev = 0.0;
    // Richardson control: saved state and the full-step result (allocated on first use)
    double *rh0 = nullptr, *rthn0 = nullptr, *rhf = nullptr;
    double err_last = 0.0, err_max = 0.0;
    int wait_polls = 0;          // test limit of the bounded device waits (0: default)

    bool closure_at_h = false;   // K[0], Can hold the closures at h (the accepted state)
    bool soils_set = false, has_state = false;
    double t = 0.0, dt_nom = 1.0;
    int easy = 0;
    long long steps = 0;
    double storage0 = 0.0, in_cum = 0.0, out_cum = 0.0, closure_cum = 0.0, defect_cum = 0.0;

    void *dalloc(size_t bytes)
    {
        bytes = (bytes + 255) & ~size_t(255);
        void *ptr = nullptr;
        if (has_alloc) ptr = alloc.alloc(bytes, alloc.user);
        else if (cudaMalloc(&ptr, bytes) != cudaSuccess) ptr = nullptr;
        if (ptr) allocations.push_back(ptr);
        return ptr;
    }
};

namespace {

template <class T>
bool alloc_n(rf_ctx *c, T *&ptr, size_t n)
{
    ptr = static_cast<T *>(c->dalloc(sizeof(T) * (n ? n : 1)));
    return ptr != nullptr;
}

rf_status check_params(const rf_solver_params *p)
{
    if (!(p->tol_picard > 0) || !(p->tol_cg > 0) || p->cg_max_it < 1 || !(p->dt0 > 0) || !(p->dt_max > 0) ||
        !(p->dt_min > 0) || !(p->f_grow >= 1.0) || !(p->f_shrink > 1.0) || p->n_inc < 1 || p->n_small < 0 ||
        p->n_max < 1 || !(p->eps_chord >= 0) || !(p->tol_inner > 0 && p->tol_inner < 1) || p->inner_max_it < 1 ||
        p->outer_max_it < 1)
        return fail(RF_ERR_ARG, "invalid solver parameters");
    if (p->precision != RF_PREC_FP64 && p->precision != RF_PREC_MIXED)
        return fail(RF_ERR_ARG, "unknown precision mode");
    if (p->precond != RF_PRECOND_JACOBI && p->precond != RF_PRECOND_MG && p->precond != RF_PRECOND_DIC &&
        p->precond != RF_PRECOND_ZLINE)
        return fail(RF_ERR_ARG, "unknown preconditioner");
    if (p->picard_form != RF_PICARD_CHORD && p->picard_form != RF_PICARD_MODIFIED)
        return fail(RF_ERR_ARG, "unknown Picard linearisation");
    if (p->precond == RF_PRECOND_MG && p->precision != RF_PREC_MIXED)
        return fail(RF_ERR_ARG, "the multigrid preconditioner serves the FP32 inner solve: use RF_PREC_MIXED");
    if (p->precond == RF_PRECOND_DIC && p->precision != RF_PREC_MIXED)
        return fail(RF_ERR_ARG, "the DIC preconditioner serves the FP32 inner solve: use RF_PREC_MIXED");
    if (p->precond == RF_PRECOND_ZLINE && p->precision != RF_PREC_MIXED)
        return fail(RF_ERR_ARG, "the vertical-line preconditioner serves the FP32 inner solve: use RF_PREC_MIXED");
    if (p->closure_arith < RF_CLOSURE_AUTO || p->closure_arith > RF_CLOSURE_DOUBLE_FLOAT)
        return fail(RF_ERR_ARG, "unknown closure arithmetic");
    if (p->face_mean != RF_FACE_ARITHMETIC && p->face_mean != RF_FACE_HARMONIC)
        return fail(RF_ERR_ARG, "unknown interface mean");
    if (p->face_mean == RF_FACE_HARMONIC && p->precision != RF_PREC_FP64)
        return fail(RF_ERR_ARG, "the harmonic interface mean runs on the FP64 path (RF_PREC_FP64)");
    if (p->time_scheme != RF_TIME_BACKWARD_EULER && p->time_scheme != RF_TIME_BDF2)
        return fail(RF_ERR_ARG, "unknown time scheme");
    if (p->time_control != RF_TIME_EBATS && p->time_control != RF_TIME_RICHARDSON)
        return fail(RF_ERR_ARG, "unknown time control");
    if (p->time_scheme == RF_TIME_BDF2 && (p->picard_form != RF_PICARD_MODIFIED || p->time_control != RF_TIME_EBATS))
        return fail(RF_ERR_ARG, "BDF2 runs in the modified Picard form under EBATS");
    if (!(p->tol_time > 0) || !std::isfinite(p->tol_time))
        return fail(RF_ERR_ARG, "tol_time (the Richardson control's bound) must be finite and > 0");
    if (!std::isfinite(p->grav[0]) || !std::isfinite(p->grav[1]) || !std::isfinite(p->grav[2]))
        return fail(RF_ERR_ARG, "non-finite gravity direction");
    return RF_OK;
}

// Grid fields that follow the solver parameters: gravity factors per face,
// the interface mean and the closure arithmetic.
void apply_grid_params(Grid &g, const rf_solver_params &p)
{
    const double gv[6] = {-p.grav[0], p.grav[0], -p.grav[1], p.grav[1], -p.grav[2], p.grav[2]};
    for (int f = 0; f < 6; f++) {
        g.gf[f] = gv[f];
        g.hg[f] = 0.5 * g.A[f] * gv[f];
    }
    g.tilted = (p.grav[0] != 0.0 || p.grav[1] != 0.0) ? 1 : 0;
    g.harmonic = p.face_mean == RF_FACE_HARMONIC ? 1 : 0;
    g.closure64 = (p.closure_arith == RF_CLOSURE_FP64 ||
                   (p.closure_arith == RF_CLOSURE_AUTO && p.precision == RF_PREC_FP64)) ? 1 : 0;
}

double series_at(const BcSeries &b, double t)
{
    size_t i = 0;
    while (i + 1 < b.v.size() && b.t[i + 1] <= t + t_tol(t)) i++;
    return b.v.empty() ? 0.0 : b.v[i];
}

double next_breakpoint(const rf_ctx *c, double t)
{
    double nb = INFINITY;
    for (int f = 0; f < 6; f++)
        for (double ti : c->bc[f].t)
            if (ti > t + t_tol(t) && ti < nb) nb = ti;
    return nb;
}

rf_status sync(rf_ctx *c)
{
    CUDA_TRY(cudaGetLastError());
    if (c->dev_fault) CUDA_TRY(cudaMemcpyAsync(c->fault_h, c->dev_fault, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->dev_fault && *c->fault_h) {
        // reported once: the flag is cleared so that the context stays usable
        *c->fault_h = 0;
        CUDA_TRY(cudaMemsetAsync(c->dev_fault, 0, sizeof(int), c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        return fail(RF_ERR_DEVICE_TIMEOUT, "a device wait for staged data ran out (the solve was stopped)");
    }
    return RF_OK;
}

// storage part of b, written and read only with modified Picard
double *s0_of(rf_ctx *c) { return c->prm.picard_form == RF_PICARD_MODIFIED ? c->s0 : nullptr; }

void fill_step_params(rf_ctx *c, double dt)
{
    StepParams &s = *c->sp_h;
    s.dt = dt;
    s.t = c->t;
    s.eps_chord = c->prm.eps_chord;
    s.modified = c->prm.picard_form == RF_PICARD_MODIFIED ? 1 : 0;
    s.bdf2 = 0;
    s.a0 = 1.0;
    s.a1 = 1.0;
    s.a2 = 0.0;
    if (c->prm.time_scheme == RF_TIME_BDF2 && c->dt_prev > 0.0) {
        const double w = dt / c->dt_prev;
        s.bdf2 = 1;
        s.a0 = (1.0 + 2.0 * w) / (1.0 + w);
        s.a1 = 1.0 + w;
        s.a2 = w * w / (1.0 + w);
    }
    for (int f = 0; f < 6; f++) {
        s.bc_type[f] = c->bc[f].type;
        s.bc_val[f] = c->bc[f].v.empty() ? 0.0 : series_at(c->bc[f], c->t);
    }
}

// Closures at h_eval (optionally with max|h_eval - hprev|) into theta_out,
// K[kout], Can.
void run_closure(rf_ctx *c, const double *h_eval, const double *hprev, double *theta_out, int kout)
{
    launch_closure(c->stream, c->nblk, c->g, c->soils, c->zone, c->Ks, c->flags, h_eval, hprev, theta_out,
                   c->K[kout], c->Can, c->partials, c->ticket, c->res);
}

void run_assemble(rf_ctx *c, const double *hk, const double *hn, const double *thk, const double *thn)
{
    launch_assemble(c->stream, c->nblk, c->g, c->soils, c->zone, c->Ks, c->flags, c->sp, hk, hn, thk, thn,
                    c->K[0], c->Can, c->c, c->b, c->Tx, c->Ty, c->Tz, c->diag, c->dinv, c->K32, c->cb32,
                    c->dinv32, nullptr, ASM_ONLY, nullptr, nullptr, nullptr, s0_of(c), c->theta_p);
}

// ---------------------------------------------------------------------------
// Graph construction.  Every loop is a conditional WHILE node whose condition
// is raised by the kernel just before it and re-set by the last kernel of its
// body on every launch (to 0 when the loop is over or was skipped), so each
// loop terminates: PCG at max_it, defect correction at outer_max_it, Picard
// at n_max.
// ---------------------------------------------------------------------------
rf_status cap_begin(rf_ctx *c, cudaGraph_t G, const std::vector<cudaGraphNode_t> &deps)
{
    CUDA_TRY(cudaStreamBeginCaptureToGraph(c->cap, G, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                           cudaStreamCaptureModeRelaxed));
    return RF_OK;
}

rf_status cap_end(rf_ctx *c, std::vector<cudaGraphNode_t> &leaves)
{
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *d = nullptr;
    size_t n = 0;
    CUDA_TRY(cudaStreamGetCaptureInfo(c->cap, &st, nullptr, nullptr, &d, nullptr, &n));
    leaves.assign(d, d + n);
    cudaGraph_t out;
    CUDA_TRY(cudaStreamEndCapture(c->cap, &out));
    CUDA_TRY(cudaGetLastError());
    return RF_OK;
}

rf_status add_while(cudaGraph_t parent, const std::vector<cudaGraphNode_t> &deps, cudaGraphConditionalHandle h,
                    cudaGraphNode_t *node, cudaGraph_t *body)
{
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    CUDA_TRY(cudaGraphAddNode(node, parent, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &np));
    *body = np.conditional.phGraph_out[0];
    return RF_OK;
}

#define RF_TRY(x)                              \
    do {                                       \
        rf_status s_ = (x);                    \
        if (s_ != RF_OK) return s_;            \
    } while (0)

// DIC arrays (allocated on first use).
rf_status ensure_dic(rf_ctx *c)
{
    if (c->dic_rd) return RF_OK;
    if (!alloc_n(c, c->dic_diag, c->g.N) || !alloc_n(c, c->dic_rd, c->g.N))
        return fail(RF_ERR_NOMEM, "DIC allocation failed");
    return RF_OK;
}

// Multigrid levels of this grid (allocated on first use).
rf_status ensure_mg(rf_ctx *c)
{
    if (c->mg_alloc) return RF_OK;
    const Grid &g = c->g;
    const double dx = g.A[0] / g.w[0], dy = g.A[2] / g.w[2], dz = g.A[4] / g.w[4];
    MgShape shp[MG_MAX_LEVELS];
    const int nl = mg_plan(g.nx, g.ny, g.nz, dx, dy, dz, shp, MG_MAX_LEVELS);
    if (nl < 2) return fail(RF_ERR_ARG, "grid too small for a multigrid hierarchy");
    MgHierarchy &H = c->mg;
    H.nlev = nl;
    for (int l = 0; l < nl; l++) {
        MgLevel &L = H.lev[l];
        L = MgLevel{};
        L.level = l;
        L.nx = shp[l].nx;
        L.ny = shp[l].ny;
        L.nz = shp[l].nz;
        L.N = (long long)L.nx * L.ny * L.nz;
        L.sxy = (long long)L.nx * L.ny;
        L.fx = make_fastdiv((unsigned int)L.nx);
        L.fxy = make_fastdiv((unsigned int)L.sxy);
        if (l + 1 < nl) {
            L.cx = shp[l + 1].nx == L.nx ? 1 : 2;
            L.cy = shp[l + 1].ny == L.ny ? 1 : 2;
            L.cz = shp[l + 1].nz == L.nz ? 1 : 2;
        } else {
            L.cx = L.cy = L.cz = 1;
        }
        const size_t n = (size_t)L.N;
        bool ok = true;
        if (l == 0) {
            L.w32[0] = g.w32[0];
            L.w32[1] = g.w32[1];
            L.w32[2] = g.w32[2];
            L.cb = c->cb32;
            L.dinv0 = c->dinv32;
            ok = alloc_n(c, L.e[1], n);
        } else {
            ok = alloc_n(c, L.cb, n) && alloc_n(c, L.T[0], n) && alloc_n(c, L.T[1], n) && alloc_n(c, L.T[2], n) &&
                 alloc_n(c, L.dinv, n) && alloc_n(c, L.r, n) && alloc_n(c, L.e[0], n) && alloc_n(c, L.e[1], n);
        }
        if (!ok) return fail(RF_ERR_NOMEM, "multigrid allocation failed");
    }
    c->mg_alloc = true;
    return RF_OK;
}

// Linear solve A x = b from x0 into x, appended to `parent` after `deps`
// (handles created on the top graph `top`).  skip: attempt-over flag or null.
// With `fused`, the assembly kernel before `deps` has already started the
// solve (x = x0, first residual, loop conditions) through `start`; otherwise
// a start kernel is captured here.  Returns the node after which the
// solution is complete.
rf_status capture_solve(rf_ctx *c, cudaGraph_t top, cudaGraph_t parent, std::vector<cudaGraphNode_t> deps,
                        const double *x0, double *x, const int *skip, bool fused, const SolveStart *start,
                        std::vector<cudaGraphNode_t> &out)
{
    const Grid &g = c->g;
    const int nb = c->nblk;
    cudaStream_t s = c->cap;
    if (c->prm.precision == RF_PREC_FP64) {
        const CondSet cc = start->cond;
        if (!fused) {
            RF_TRY(cap_begin(c, parent, deps));
            launch_cg64_init(s, nb, g, c->flags, x0, x, c->b, c->Tx, c->Ty, c->Tz, c->diag, c->dinv, c->r, c->z,
                             c->prm.tol_cg, c->prm.cg_max_it, c->partials, c->ticket, c->sc, skip, cc);
            RF_TRY(cap_end(c, deps));
        }
        cudaGraphNode_t wn;
        cudaGraph_t body;
        RF_TRY(add_while(parent, deps, cc.h, &wn, &body));
        RF_TRY(cap_begin(c, body, {}));
        for (int half = 0; half < 2; half++) {
            double *pin = c->p[half], *pout = c->p[half ^ 1];
            launch_cg64_spmv(s, nb, g, c->flags, c->z, pin, pout, c->q, c->Tx, c->Ty, c->Tz, c->diag, c->partials,
                             c->ticket, c->sc);
            launch_cg64_update(s, nb, g, x, c->r, c->z, pout, c->q, c->dinv, c->partials, c->ticket, c->sc, cc);
        }
        std::vector<cudaGraphNode_t> tmp;
        RF_TRY(cap_end(c, tmp));
        out = {wn};
        return RF_OK;
    }
    // mixed: WHILE(outer) { WHILE(inner FP32 PCG) ; x += d ; FP64 residual }
    const CondSet co = start->cond, ci = start->cond_inner;
    const bool mg = c->prm.precond == RF_PRECOND_MG, dic = c->prm.precond == RF_PRECOND_DIC;
    const int *idone = &c->sc_in->done;
    // z = M r for the MG preconditioner
    auto precondition = [&]() { launch_mg_vcycle(s, nb, c->mg, c->K32, c->r32, c->z32, idone); };
    const CondSet none{0, 0};
    if (!fused) {
        RF_TRY(cap_begin(c, parent, deps));
        launch_mixed_start(s, nb, g, x0, x, c->sc, c->sc_in, skip, co);
        launch_resid64(s, nb, g, c->flags, x, c->b, c->Tx, c->Ty, c->Tz, c->diag, c->dinv32, c->r32, c->z32, c->d32,
                       c->prm.tol_cg, c->prm.tol_inner, c->prm.inner_max_it, c->prm.outer_max_it, c->partials,
                       c->ticket, c->sc, c->sc_in, co, ci);
        RF_TRY(cap_end(c, deps));
    }
    // z = M r and rho = r.z (start) or beta (inner iterations); DIC folds
    // r.z into its two sweeps, and within the loop its red pass into the update
    auto precondition_rz = [&](int first, bool red_done) {
        if (dic) {
            launch_dic_apply_rz(s, nb, g, c->K32, c->dic_rd, c->r32, c->z32, c->partials, c->ticket, c->sc_in,
                                first, red_done, ci);
        } else {
            precondition();
            launch_cg32_rz(s, nb, g, c->r32, c->z32, c->partials, c->ticket, c->sc_in, first, ci);
        }
    };
    if (mg || dic) {
        // coarse operators (MG) or pivots (DIC) from this assembly, then
        // z0 = M r0 and rho = r0.z0
        RF_TRY(cap_begin(c, parent, deps));
        if (mg) launch_mg_build(s, nb, c->mg, c->K32, skip);
        else launch_dic_setup(s, nb, g, c->K32, c->cb32, c->dic_diag, c->dic_rd, skip);
        precondition_rz(1, false);
        RF_TRY(cap_end(c, deps));
    }
    cudaGraphNode_t wo, wi;
    cudaGraph_t bo, bi;
    RF_TRY(add_while(parent, deps, co.h, &wo, &bo));
    RF_TRY(add_while(bo, {}, ci.h, &wi, &bi));
    RF_TRY(cap_begin(c, bi, {}));
    for (int half = 0; half < 2; half++) {
        float *pin = c->p32[half], *pout = c->p32[half ^ 1];
        launch_cg32_spmv(s, nb, g, c->z32, pin, pout, c->q32, c->K32, c->cb32, c->partials, c->ticket, c->sc_in,
                         c->tma_ok ? &c->tma : nullptr, c->dev_fault);
        if (dic) {
            launch_cg32_update_dic(s, nb, g, c->d32, c->r32, c->z32, pout, c->q32, c->dinv32, c->dic_rd, c->partials,
                                   c->ticket, c->sc_in);
            precondition_rz(0, true);
        } else if (mg) {
            launch_cg32_update_mg(s, nb, g, c->d32, c->r32, pout, c->q32, c->dinv32, c->partials, c->ticket, c->sc_in);
            precondition_rz(0, false);
        } else {
            launch_cg32_update(s, nb, g, c->d32, c->r32, c->z32, pout, c->q32, c->dinv32, c->partials, c->ticket,
                               c->sc_in, ci);
        }
    }
    std::vector<cudaGraphNode_t> tmp;
    RF_TRY(cap_end(c, tmp));
    RF_TRY(cap_begin(c, bo, {wi}));
    launch_add_correction(s, nb, g, x, c->d32, c->sc, c->sc_in, co);
    launch_resid64(s, nb, g, c->flags, x, c->b, c->Tx, c->Ty, c->Tz, c->diag, c->dinv32, c->r32, c->z32, c->d32,
                   c->prm.tol_cg, c->prm.tol_inner, c->prm.inner_max_it, c->prm.outer_max_it, c->partials, c->ticket,
                   c->sc, c->sc_in, co, ci);
    if (mg || dic) precondition_rz(1, false);
    (void)none;
    RF_TRY(cap_end(c, tmp));
    out = {wo};
    return RF_OK;
}

// Loop handles and start description of one linear solve in graph G.
rf_status make_start(rf_ctx *c, cudaGraph_t G, double *x, SolveStart &st)
{
    st = SolveStart{};
    cudaGraphConditionalHandle h1, h2;
    CUDA_TRY(cudaGraphConditionalHandleCreate(&h1, G, 0, 0));
    st.cond = CondSet{h1, 1};
    if (c->prm.precision == RF_PREC_MIXED) {
        CUDA_TRY(cudaGraphConditionalHandleCreate(&h2, G, 0, 0));
        st.cond_inner = CondSet{h2, 1};
    }
    st.x = x;
    st.r = c->r;
    st.z = c->z;
    st.r32 = c->r32;
    st.z32 = c->z32;
    st.d32 = c->d32;
    st.sc = c->sc;
    st.inner = c->sc_in;
    st.tol = c->prm.tol_cg;
    st.tol_inner = c->prm.tol_inner;
    st.max_it = c->prm.cg_max_it;
    st.inner_max_it = c->prm.inner_max_it;
    st.outer_max_it = c->prm.outer_max_it;
    return RF_OK;
}

void destroy_graphs(rf_ctx *c)
{
    if (c->picard_exec) cudaGraphExecDestroy(c->picard_exec);
    if (c->picard_graph) cudaGraphDestroy(c->picard_graph);
    if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
    if (c->solve_graph) cudaGraphDestroy(c->solve_graph);
    c->picard_exec = nullptr;
    c->picard_graph = nullptr;
    c->solve_exec = nullptr;
    c->solve_graph = nullptr;
}

// One Picard attempt as a graph: WHILE(Picard) { half A ; half B }, where a
// half is assemble -> linear solve -> closures + exit test -> water balance,
// half A iterating h^k = H0 -> x = H1 (K0 -> K1) and half B the reverse, so
// the buffers never move.  Kernels of a half that starts after the attempt
// ended return at once.
rf_status build_picard_graph(rf_ctx *c)
{
    if (c->prm.precond == RF_PRECOND_MG) RF_TRY(ensure_mg(c));
    if (c->prm.precond == RF_PRECOND_DIC) RF_TRY(ensure_dic(c));
    cudaGraph_t G;
    CUDA_TRY(cudaGraphCreate(&G, 0));
    c->picard_graph = G;
    cudaGraphConditionalHandle hp;
    CUDA_TRY(cudaGraphConditionalHandleCreate(&hp, G, 1, cudaGraphCondAssignDefault));
    const CondSet cp{hp, 1};
    cudaGraphNode_t wp;
    cudaGraph_t body;
    RF_TRY(add_while(G, {}, hp, &wp, &body));
    const Grid &g = c->g;
    const int nb = c->nblk;
    cudaStream_t s = c->cap;
    const int *skip = &c->ctl->done;
    double *H[2] = {c->hk, c->x};
    std::vector<cudaGraphNode_t> deps;
    for (int half = 0; half < 2; half++) {
        double *hk = H[half], *x = H[half ^ 1];
        double *Kin = c->K[half], *Kout = c->K[half ^ 1];
        SolveStart st;
        RF_TRY(make_start(c, G, x, st));
        RF_TRY(cap_begin(c, body, deps));
        launch_assemble(s, nb, g, c->soils, c->zone, c->Ks, c->flags, c->sp, hk, c->h, c->theta_k, c->theta_n, Kin,
                        c->Can, c->c, c->b, c->Tx, c->Ty, c->Tz, c->diag, c->dinv, c->K32, c->cb32, c->dinv32, skip,
                        c->prm.precision == RF_PREC_FP64 ? ASM_CG64 : ASM_MIXED, &st, c->partials, c->ticket,
                        s0_of(c), c->theta_p);
        RF_TRY(cap_end(c, deps));
        RF_TRY(capture_solve(c, G, body, deps, hk, x, skip, true, &st, deps));
        RF_TRY(cap_begin(c, body, deps));
        const CgScal *stat = c->sc;   // FP64 solve, or outer defect-correction loop
        const CgScal *cnt = c->prm.precision == RF_PREC_FP64 ? c->sc : c->sc_in;
        launch_closure_picard(s, nb, g, c->soils, c->zone, c->Ks, c->flags, x, hk, c->theta_k, Kout, c->Can,
                              c->partials, c->ticket, c->ctl, stat, cnt, cp);
        RF_TRY(cap_end(c, deps));
    }
    // water balance of the converged system, once, after the Picard loop: an
    // odd iteration count ends in half 0 (iterate in x, system K in K[0]),
    // an even one in half 1 (iterate in hk, K[1])
    std::vector<cudaGraphNode_t> after;
    RF_TRY(cap_begin(c, G, {wp}));
    launch_mass_balance(s, nb, g, c->soils, c->zone, c->Ks, c->flags, c->sp, c->x, c->hk, c->h, c->c, c->K[0],
                        c->K[1], c->theta_k, c->theta_n, c->partials, c->ticket, c->res, c->ctl, s0_of(c));
    RF_TRY(cap_end(c, after));
    CUDA_TRY(cudaGraphInstantiate(&c->picard_exec, G, 0));
    return RF_OK;
}

rf_status build_solve_graph(rf_ctx *c)
{
    if (c->prm.precond == RF_PRECOND_MG) RF_TRY(ensure_mg(c));
    if (c->prm.precond == RF_PRECOND_DIC) RF_TRY(ensure_dic(c));
    cudaGraph_t G;
    CUDA_TRY(cudaGraphCreate(&G, 0));
    c->solve_graph = G;
    std::vector<cudaGraphNode_t> out;
    SolveStart st;
    RF_TRY(make_start(c, G, c->x, st));
    RF_TRY(capture_solve(c, G, G, {}, c->hk, c->x, nullptr, false, &st, out));
    CUDA_TRY(cudaGraphInstantiate(&c->solve_exec, G, 0));
    return RF_OK;
}

// Solve the assembled system from hk into x (kernel-level entry point).
rf_status solve_system(rf_ctx *c, int *iters)
{
    if (!c->solve_exec) RF_TRY(build_solve_graph(c));
    CUDA_TRY(cudaGraphLaunch(c->solve_exec, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->sc_h, c->sc, sizeof(CgScal), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->sc_in_h, c->sc_in, sizeof(CgScal), cudaMemcpyDeviceToHost, c->stream));
    RF_TRY(sync(c));
    *iters = c->prm.precision == RF_PREC_FP64 ? c->sc_h->total : c->sc_in_h->total;
    if (c->sc_h->status != CG_OK)
        return fail(RF_ERR_CG, c->sc_h->status == CG_MAXIT ? "linear solve reached its iteration cap" : "non-finite linear solve");
    return RF_OK;
}

struct Attempt {
    bool converged = false;
    int picard = 0, cg = 0;
    rf_status status = RF_OK;
    double max_dh = 0.0;
    StepResults mb{};
};

// One Picard attempt at step size dt from the accepted state h (Sec. 2.2),
// run on the device as one graph launch; one host synchronisation.
// Feature values of the top flux and the step size (the scalar features).
void ws_scalar_features(const rf_ctx *c, const nn::WsScales &sc, double t, double dt, float &q_feat, float &dt_feat)
{
    const BcSeries &top = c->bc[F_ZMAX];
    const double q = (top.type == BC_FLUX && !top.v.empty()) ? series_at(top, t) : 0.0;
    q_feat = (float)(q / sc.q_scale);
    dt_feat = (float)std::log(dt / sc.t_scale);
}

rf_status attempt(rf_ctx *c, double dt, Attempt &A, bool guess)
{
    NvtxRange range("rf: Picard attempt");
    if (!c->picard_exec) RF_TRY(build_picard_graph(c));
    fill_step_params(c, dt);
    PicardCtl &ctl = *c->ctl_h;
    ctl = PicardCtl{};
    ctl.tol = c->prm.tol_picard;
    ctl.n_max = c->prm.n_max;
    CUDA_TRY(cudaMemcpyAsync(c->sp, c->sp_h, sizeof(StepParams), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->ctl, c->ctl_h, sizeof(PicardCtl), cudaMemcpyHostToDevice, c->stream));
    if (guess) {
        // first iterate from the network: hk = h + y out_scale dt, closures at hk
        float q_feat, dt_feat;
        ws_scalar_features(c, c->ws_sc, c->t, dt, q_feat, dt_feat);
        RF_TRY(rf_nn_mesh_guess(c->ws_net, c->stream, c->g, c->flags, c->h, c->Ks, c->ws_sc, q_feat, dt_feat,
                                c->ws_sc.out_scale * dt, c->hk, c->dev_fault));
        run_closure(c, c->hk, nullptr, c->theta_k, 0);
        c->closure_at_h = false;
        c->ws_guesses++;
    } else {
        CUDA_TRY(cudaMemcpyAsync(c->hk, c->h, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice, c->stream));
        if (!c->closure_at_h) {
            run_closure(c, c->hk, nullptr, c->theta_k, 0);
            c->closure_at_h = true;
        }
    }
    CUDA_TRY(cudaGraphLaunch(c->picard_exec, c->stream));
    c->closure_at_h = false;     // the attempt overwrites K[0] and C; an accepted step sets it again
    CUDA_TRY(cudaMemcpyAsync(c->ctl_h, c->ctl, sizeof(PicardCtl), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->res_h, c->res, sizeof(StepResults), cudaMemcpyDeviceToHost, c->stream));
    RF_TRY(sync(c));
    A.picard = ctl.it;
    A.cg = ctl.cg_total;
    A.max_dh = ctl.max_dh;
    if (ctl.conv) {
        A.converged = true;
        A.mb = *c->res_h;
        // the last iterate and its closures: H[it & 1], K[it & 1]
        const int f = ctl.it & 1;
        if (c->prm.time_scheme == RF_TIME_BDF2)    // theta*(h^{n-1}) for the next step
            CUDA_TRY(cudaMemcpyAsync(c->theta_p, c->theta_n, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice,
                                     c->stream));
        launch_accept(c->stream, c->nblk, c->g, f ? c->x : c->hk, c->h, c->theta_k, c->theta_n, c->K[1], c->K[0], f);
    } else {
        A.status = ctl.fail ? RF_ERR_CG : RF_ERR_PICARD;
        if (guess) c->ws_fallbacks++;
    }
    return RF_OK;
}

void ebats_accept(rf_ctx *c, int picard)
{
    if (picard <= c->prm.n_small) c->easy++;
    else c->easy = 0;
    if (c->easy >= c->prm.n_inc) {
        c->dt_nom = std::min(c->dt_nom * c->prm.f_grow, c->prm.dt_max);
        c->easy = 0;
    }
}

// One accepted step with EBATS reruns, clipped to t_stop.
rf_status do_step(rf_ctx *c, double t_stop, rf_step_info *info)
{
    if (!c->soils_set || !c->has_state) return fail(RF_ERR_STATE, "set soils and state before stepping");
    const double dt_nom0 = c->dt_nom;
    const int easy0 = c->easy;
    int rejected = 0, cg_total = 0;
    for (;;) {
        double dt = c->dt_nom;
        const double bp = next_breakpoint(c, c->t);
        if (bp - c->t < dt) dt = bp - c->t;
        if (t_stop - c->t < dt) dt = t_stop - c->t;
        Attempt A;
        // a rejected attempt from the guess falls back to the plain start
        rf_status st = attempt(c, dt, A, c->ws_net != nullptr && rejected == 0);
        if (st) { c->dt_nom = dt_nom0; c->easy = easy0; return st; }
        cg_total += A.cg;
        if (A.converged) {
            c->closure_at_h = true;
            if (c->prm.time_scheme == RF_TIME_BDF2) c->dt_prev = dt;
            double tn = c->t + dt;
            if (std::fabs(tn - bp) <= t_tol(tn)) tn = bp;
            if (std::fabs(tn - t_stop) <= t_tol(tn)) tn = t_stop;
            c->t = tn;
            c->steps++;
            const double net = A.mb.bnd_in - A.mb.bnd_out;
            c->in_cum += A.mb.bnd_in;
            c->out_cum += A.mb.bnd_out;
            c->closure_cum += A.mb.lin_change - net;
            c->defect_cum += A.mb.dstore - net;
            ebats_accept(c, A.picard);
            if (info) {
                info->dt = dt;
                info->t = c->t;
                info->picard_iters = A.picard;
                info->cg_iters = cg_total;
                info->rejected = rejected;
                info->max_dh = A.max_dh;
            }
            return RF_OK;
        }
        rejected++;
        c->dt_nom = dt / c->prm.f_shrink;
        c->easy = 0;
        if (c->dt_nom < c->prm.dt_min) {
            c->dt_nom = dt_nom0;
            c->easy = easy0;
            return fail(RF_ERR_DT_MIN, "EBATS: dt fell below dt_min without Picard convergence at t = " +
                                           std::to_string(c->t));
        }
    }
}

// Richardson step doubling (the alternative to EBATS that Sec. 2.2 names for
// prescribing the temporal error).  Each step runs once with dt and twice
// with dt/2 from the same state; the local error estimate is max over active
// cells |h(2 x dt/2) - h(dt)|; the step is accepted, with the two-half-step
// result, when the estimate is within tol_time.  The next dt is
// dt 0.9 sqrt(tol_time / err) clamped to [0.2, 2] dt and to dt_max either way;
// a Picard failure in any of the three solves divides dt by f_shrink as in
// EBATS.  attempt() accepts a converged solve into h, theta_n and K[0], so the
// state at the step start is saved and put back around each solve.
rf_status ensure_richardson(rf_ctx *c)
{
    if (c->rh0) return RF_OK;
    if (!alloc_n(c, c->rh0, c->g.N) || !alloc_n(c, c->rthn0, c->g.N) || !alloc_n(c, c->rhf, c->g.N))
        return fail(RF_ERR_NOMEM, "Richardson control: device allocation failed");
    return RF_OK;
}

rf_status richardson_restore(rf_ctx *c)
{
    const size_t nb = sizeof(double) * c->g.N;
    CUDA_TRY(cudaMemcpyAsync(c->h, c->rh0, nb, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->theta_n, c->rthn0, nb, cudaMemcpyDeviceToDevice, c->stream));
    c->closure_at_h = false;
    return RF_OK;
}

rf_status do_step_richardson(rf_ctx *c, double t_stop, rf_step_info *info)
{
    NvtxRange range("rf: Richardson step");
    if (!c->soils_set || !c->has_state) return fail(RF_ERR_STATE, "set soils and state before stepping");
    RF_TRY(ensure_richardson(c));
    const double dt_nom0 = c->dt_nom, t0 = c->t;
    const size_t nb = sizeof(double) * c->g.N;
    CUDA_TRY(cudaMemcpyAsync(c->rh0, c->h, nb, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->rthn0, c->theta_n, nb, cudaMemcpyDeviceToDevice, c->stream));
    int rejected = 0, cg_total = 0, pic_total = 0;
    // on an error: the state at the step start, time and dt_nom put back
    auto abort = [&](rf_status st) {
        const std::string msg = g_err;
        richardson_restore(c);
        cudaStreamSynchronize(c->stream);
        c->t = t0;
        c->dt_nom = dt_nom0;
        g_err = msg;
        return st;
    };
    for (;;) {
        double dt = c->dt_nom;
        const double bp = next_breakpoint(c, t0);
        if (bp - t0 < dt) dt = bp - t0;
        if (t_stop - t0 < dt) dt = t_stop - t0;
        Attempt Af, A1, A2;
        c->t = t0;
        if (rf_status st = attempt(c, dt, Af, false)) return abort(st);
        cg_total += Af.cg;
        pic_total += Af.picard;
        bool ok = Af.converged;
        if (ok) {
            CUDA_TRY(cudaMemcpyAsync(c->rhf, c->h, nb, cudaMemcpyDeviceToDevice, c->stream));
            RF_TRY(richardson_restore(c));
            if (rf_status st = attempt(c, 0.5 * dt, A1, false)) return abort(st);
            cg_total += A1.cg;
            pic_total += A1.picard;
            ok = A1.converged;
        }
        if (ok) {
            c->t = t0 + 0.5 * dt;
            if (rf_status st = attempt(c, 0.5 * dt, A2, false)) return abort(st);
            c->t = t0;
            cg_total += A2.cg;
            pic_total += A2.picard;
            ok = A2.converged;
        }
        if (!ok) {
            RF_TRY(richardson_restore(c));
            rejected++;
            c->dt_nom = dt / c->prm.f_shrink;
            if (c->dt_nom < c->prm.dt_min) {
                c->dt_nom = dt_nom0;
                return fail(RF_ERR_DT_MIN, "Richardson control: dt fell below dt_min without Picard convergence at t = " +
                                               std::to_string(t0));
            }
            continue;
        }
        // h holds h(2 x dt/2): its closures (kept for the next step) and the
        // error estimate max |h - h(dt)| in one pass
        run_closure(c, c->h, c->rhf, c->theta_k, 0);
        CUDA_TRY(cudaMemcpyAsync(c->res_h, c->res, sizeof(StepResults), cudaMemcpyDeviceToHost, c->stream));
        if (rf_status st = sync(c)) return abort(st);
        const double err = c->res_h->nonfinite ? INFINITY : c->res_h->max_dh;
        double fac = err > 0.0 ? 0.9 * std::sqrt(c->prm.tol_time / err) : 2.0;
        fac = std::min(2.0, std::max(0.2, fac));
        c->dt_nom = std::min(dt * fac, c->prm.dt_max);
        c->err_last = err;
        if (!(err <= c->prm.tol_time)) {
            RF_TRY(richardson_restore(c));
            rejected++;
            if (c->dt_nom < c->prm.dt_min) {
                c->dt_nom = dt_nom0;
                return fail(RF_ERR_DT_MIN, "Richardson control: dt fell below dt_min at t = " + std::to_string(t0));
            }
            continue;
        }
        c->closure_at_h = true;
        c->err_max = std::max(c->err_max, err);
        double tn = t0 + dt;
        if (std::fabs(tn - bp) <= t_tol(tn)) tn = bp;
        if (std::fabs(tn - t_stop) <= t_tol(tn)) tn = t_stop;
        c->t = tn;
        c->steps++;
        c->in_cum += A1.mb.bnd_in + A2.mb.bnd_in;
        c->out_cum += A1.mb.bnd_out + A2.mb.bnd_out;
        c->closure_cum += (A1.mb.lin_change - (A1.mb.bnd_in - A1.mb.bnd_out)) +
                          (A2.mb.lin_change - (A2.mb.bnd_in - A2.mb.bnd_out));
        c->defect_cum += (A1.mb.dstore - (A1.mb.bnd_in - A1.mb.bnd_out)) +
                         (A2.mb.dstore - (A2.mb.bnd_in - A2.mb.bnd_out));
        if (info) {
            info->dt = dt;
            info->t = c->t;
            info->picard_iters = pic_total;
            info->cg_iters = cg_total;
            info->rejected = rejected;
            info->max_dh = A2.max_dh;
        }
        return RF_OK;
    }
}

// One accepted step under the context's time control.
rf_status step_any(rf_ctx *c, double t_stop, rf_step_info *info)
{
    return c->prm.time_control == RF_TIME_RICHARDSON ? do_step_richardson(c, t_stop, info) : do_step(c, t_stop, info);
}

rf_status storage_of_theta_n(rf_ctx *c, double *out)
{
    launch_storage(c->stream, c->nblk, c->g, c->flags, c->theta_n, c->partials, c->ticket, c->res);
    CUDA_TRY(cudaMemcpyAsync(c->res_h, c->res, sizeof(StepResults), cudaMemcpyDeviceToHost, c->stream));
    rf_status st = sync(c);
    if (st) return st;
    *out = c->res_h->storage;
    return RF_OK;
}

}  // namespace

namespace rf {
// rf_solver_params validation, shared with rf_ens_create
rf_status check_solver_params(const rf_solver_params *p) { return check_params(p); }
}  // namespace rf

// =========================================================================
extern "C" {

void rf_default_params(rf_solver_params *p)
{
    if (!p) return;
    p->tol_picard = 1e-6;
    p->tol_cg = 1e-10;
    p->cg_max_it = 10000;
    p->precond = RF_PRECOND_JACOBI;
    p->precision = RF_PREC_FP64;
    p->dt0 = 1.0;
    p->dt_max = 600.0;
    p->dt_min = 1e-3;
    p->f_grow = 1.3;
    p->f_shrink = 1.3;
    p->n_inc = 10;
    p->n_small = 3;
    p->n_max = 8;
    p->eps_chord = 1e-10;
    p->tol_inner = 1e-4;
    p->inner_max_it = 2000;
    p->outer_max_it = 30;
    p->picard_form = RF_PICARD_CHORD;
    p->closure_arith = RF_CLOSURE_AUTO;
    p->face_mean = RF_FACE_ARITHMETIC;
    p->time_scheme = RF_TIME_BACKWARD_EULER;
    p->time_control = RF_TIME_EBATS;
    p->tol_time = 1e-3;
    p->grav[0] = 0.0;
    p->grav[1] = 0.0;
    p->grav[2] = 1.0;
}

const char *rf_last_error(void) { return g_err.c_str(); }

rf_status rf_mesh_create(const rf_mesh_desc *mesh, const rf_solver_params *params, void *cuda_stream,
                         const rf_allocator *alloc, rf_ctx **out)
{
    if (out) *out = nullptr;
    if (!mesh || !out) return fail(RF_ERR_ARG, "null argument");
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || !(mesh->dx > 0) || !(mesh->dy > 0) || !(mesh->dz > 0))
        return fail(RF_ERR_ARG, "mesh sizes and spacings must be positive");
    const long long N = (long long)mesh->nx * mesh->ny * mesh->nz;
    if (N > (1LL << 31) - 1) return fail(RF_ERR_ARG, "mesh too large (more than 2^31-1 cells)");
    rf_solver_params prm;
    rf_default_params(&prm);
    if (params) prm = *params;
    if (rf_status st = check_params(&prm)) return st;
    if (prm.precond == RF_PRECOND_ZLINE)
        return fail(RF_ERR_ARG, "the vertical-line preconditioner serves the ensemble (rf_ens_create) only");

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return fail(RF_ERR_NO_DEVICE, "no CUDA device visible; this library has no CPU fallback");
    }
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    if (prop.major != 10 || prop.minor != 3)
        return fail(RF_ERR_NO_DEVICE, std::string("device is sm_") + std::to_string(prop.major * 10 + prop.minor) +
                                          "; this library is built for sm_103a (GB300) only");

    rf_ctx *c = new rf_ctx();
    c->device = dev;
    c->num_sms = prop.multiProcessorCount;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (alloc && alloc->alloc && alloc->free) { c->alloc = *alloc; c->has_alloc = true; }
    c->prm = prm;

    Grid &g = c->g;
    g.nx = mesh->nx; g.ny = mesh->ny; g.nz = mesh->nz;
    g.N = N;
    g.sxy = (long long)mesh->nx * mesh->ny;
    g.V = mesh->dx * mesh->dy * mesh->dz;
    const double A[6] = {mesh->dy * mesh->dz, mesh->dy * mesh->dz, mesh->dx * mesh->dz, mesh->dx * mesh->dz,
                         mesh->dx * mesh->dy, mesh->dx * mesh->dy};
    const double d[6] = {mesh->dx, mesh->dx, mesh->dy, mesh->dy, mesh->dz, mesh->dz};
    for (int f = 0; f < 6; f++) {
        g.A[f] = A[f];
        g.w[f] = A[f] / d[f];
        g.wb[f] = A[f] / (0.5 * d[f]);
        g.hw[f] = 0.5 * (A[f] / d[f]);
    }
    apply_grid_params(g, prm);
    for (int a = 0; a < 3; a++) g.w32[a] = (float)(A[2 * a] / d[2 * a]);
    g.fx = make_fastdiv((unsigned int)g.nx);
    g.fxy = make_fastdiv((unsigned int)g.sxy);
    // grid: at most 8 resident blocks of 256 threads per SM
    const long long want = (N + RED_THREADS - 1) / RED_THREADS;
    c->nblk = (int)std::max(1LL, std::min(want, (long long)c->num_sms * 8));
    g.cap = std::max(c->nblk, c->num_sms * 8);

    // flags: active bit + boundary faces (domain edge, or a z-face whose
    // neighbour is inactive); lateral faces touching an inactive cell are closed
    c->flags_h.assign(N, 0);
    auto act = [&](long long p) { return mesh->active ? mesh->active[p] != 0 : true; };
    for (int k = 0; k < g.nz; k++)
        for (int j = 0; j < g.ny; j++)
            for (int i = 0; i < g.nx; i++) {
                const long long p = i + (long long)g.nx * (j + (long long)g.ny * k);
                if (!act(p)) continue;
                uint8_t fl = FLAG_ACTIVE;
                if (i == 0) fl |= 1u << F_XMIN;
                if (i == g.nx - 1) fl |= 1u << F_XMAX;
                if (j == 0) fl |= 1u << F_YMIN;
                if (j == g.ny - 1) fl |= 1u << F_YMAX;
                if (k == 0 || !act(p - g.sxy)) fl |= 1u << F_ZMIN;
                if (k == g.nz - 1 || !act(p + g.sxy)) fl |= 1u << F_ZMAX;
                c->flags_h[p] = fl;
                c->n_active++;
            }

    bool ok = alloc_n(c, c->flags, N) && alloc_n(c, c->zone, N) && alloc_n(c, c->Ks, N) &&
              alloc_n(c, c->soils, 256) && alloc_n(c, c->h, N) && alloc_n(c, c->hk, N) && alloc_n(c, c->x, N) &&
              alloc_n(c, c->theta_n, N) && alloc_n(c, c->theta_k, N) && alloc_n(c, c->K[0], N) &&
              alloc_n(c, c->K[1], N) && alloc_n(c, c->Can, N) && alloc_n(c, c->c, N) && alloc_n(c, c->b, N) &&
              (c->prm.picard_form != RF_PICARD_MODIFIED || alloc_n(c, c->s0, N)) &&
              (c->prm.time_scheme != RF_TIME_BDF2 || alloc_n(c, c->theta_p, N)) &&
              alloc_n(c, c->Tx, N) && alloc_n(c, c->Ty, N) && alloc_n(c, c->Tz, N) && alloc_n(c, c->diag, N) &&
              alloc_n(c, c->dinv, N) && alloc_n(c, c->r, N) && alloc_n(c, c->z, N) && alloc_n(c, c->p[0], N) &&
              alloc_n(c, c->p[1], N) && alloc_n(c, c->q, N) && alloc_n(c, c->K32, N) && alloc_n(c, c->cb32, N) &&
              alloc_n(c, c->dinv32, N) && alloc_n(c, c->r32, N) && alloc_n(c, c->z32, N) &&
              alloc_n(c, c->p32[0], N) && alloc_n(c, c->p32[1], N) && alloc_n(c, c->q32, N) &&
              alloc_n(c, c->d32, N) && alloc_n(c, c->partials, (size_t)8 * g.cap) && alloc_n(c, c->ticket, 64) &&
              alloc_n(c, c->sc, 1) && alloc_n(c, c->sc_in, 1) && alloc_n(c, c->res, 1) && alloc_n(c, c->sp, 1) &&
              alloc_n(c, c->ctl, 1) && alloc_n(c, c->ctr, 2 * KK_COUNT) && alloc_n(c, c->fftab, 1) &&
              alloc_n(c, c->dev_fault, 1);
    if (!ok) {
        rf_destroy(c);
        return fail(RF_ERR_NOMEM, "device allocation failed");
    }
    if (cudaMallocHost(&c->sc_h, sizeof(CgScal)) != cudaSuccess ||
        cudaMallocHost(&c->sc_in_h, sizeof(CgScal)) != cudaSuccess ||
        cudaMallocHost(&c->res_h, sizeof(StepResults)) != cudaSuccess ||
        cudaMallocHost(&c->sp_h, sizeof(StepParams)) != cudaSuccess ||
        cudaMallocHost(&c->ctl_h, sizeof(PicardCtl)) != cudaSuccess ||
        cudaMallocHost(&c->ctr_h, 2 * KK_COUNT * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&c->fault_h, sizeof(int)) != cudaSuccess) {
        rf_destroy(c);
        return fail(RF_ERR_NOMEM, "pinned host allocation failed");
    }
    if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
        rf_destroy(c);
        return fail(RF_ERR_CUDA, "capture stream creation failed");
    }
    g.ctr = c->ctr;
    g.tab = c->fftab;
    FFTables tab;
    make_ff_tables(&tab);
    cudaError_t e = cudaMemcpyAsync(c->flags, c->flags_h.data(), N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->fftab, &tab, sizeof(FFTables), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ticket, 0, 64 * sizeof(unsigned int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ctr, 0, 2 * KK_COUNT * sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ctl, 0, sizeof(PicardCtl), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dev_fault, 0, sizeof(int), c->stream);
    // vectors whose inactive entries must read as zero
    for (double *v : {c->p[0], c->p[1], c->q, c->r, c->z, c->h, c->hk, c->x})
        if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, sizeof(double) * N, c->stream);
    for (float *v : {c->p32[0], c->p32[1], c->q32, c->r32, c->z32, c->d32})
        if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, sizeof(float) * N, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        rf_destroy(c);
        return fail(RF_ERR_CUDA, std::string("initialisation: ") + cudaGetErrorString(e));
    }
    // TMA plane staging for the FP32 stencil (grids with nx a multiple of 4)
    c->tma_ok = make_tma_maps32(g.nx, g.ny, g.nz, c->z32, c->p32[0], c->p32[1], c->K32, c->cb32, &c->tma);
    cudaGetLastError();
    *out = c;
    return RF_OK;
}

void rf_destroy(rf_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    destroy_graphs(c);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (void *ptr : c->allocations) {
        if (c->has_alloc) c->alloc.free(ptr, c->alloc.user);
        else cudaFree(ptr);
    }
    if (c->fault_h) cudaFreeHost(c->fault_h);
    if (c->sc_h) cudaFreeHost(c->sc_h);
    if (c->sc_in_h) cudaFreeHost(c->sc_in_h);
    if (c->res_h) cudaFreeHost(c->res_h);
    if (c->sp_h) cudaFreeHost(c->sp_h);
    if (c->ctl_h) cudaFreeHost(c->ctl_h);
    if (c->ctr_h) cudaFreeHost(c->ctr_h);
    delete c;
}

rf_status rf_set_params(rf_ctx *c, const rf_solver_params *params)
{
    if (!c || !params) return fail(RF_ERR_ARG, "null argument");
    if (rf_status st = check_params(params)) return st;
    if (params->precond == RF_PRECOND_ZLINE)
        return fail(RF_ERR_ARG, "the vertical-line preconditioner serves the ensemble (rf_ens_create) only");
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (params->picard_form == RF_PICARD_MODIFIED && !c->s0 && !alloc_n(c, c->s0, c->g.N))
        return fail(RF_ERR_NOMEM, "rf_set_params: device allocation failed");
    if (params->time_scheme == RF_TIME_BDF2 && !c->theta_p && !alloc_n(c, c->theta_p, c->g.N))
        return fail(RF_ERR_NOMEM, "rf_set_params: device allocation failed");
    destroy_graphs(c);   // tolerances, caps and grid fields are baked into the graphs
    if (params->time_scheme != c->prm.time_scheme) c->dt_prev = 0.0;   // no BDF2 history across a switch
    c->prm = *params;
    apply_grid_params(c->g, c->prm);
    c->closure_at_h = false;   // the closure arithmetic may have changed
    return RF_OK;
}

rf_status rf_soil_set(rf_ctx *c, const rf_soil *zones, int n_zones, const uint8_t *zone_of_cell,
                      const double *Ks_cell)
{
    if (!c || !zones || n_zones < 1 || n_zones > 256) return fail(RF_ERR_ARG, "need 1..256 soil zones");
    std::vector<DevSoil> soils(256);
    for (int z = 0; z < n_zones; z++) {
        const rf_soil &s = zones[z];
        if ((s.model != RF_VG && s.model != RF_GARDNER && s.model != RF_BROOKS_COREY) || !(s.theta_s > s.theta_r) ||
            !(s.alpha > 0) || !(s.Ks > 0) || !(s.S >= 0) || (s.model == RF_VG && !(s.n > 1.0)) ||
            (s.model == RF_BROOKS_COREY && !(s.n > 0.0)))
            return fail(RF_ERR_ARG, "invalid soil parameters in zone " + std::to_string(z));
        const double m = s.model == RF_VG ? 1.0 - 1.0 / s.n : 0.0;
        const float nh = (float)s.n, mh = (float)m;
        soils[z] = DevSoil{s.model, s.theta_r, s.theta_s, s.alpha, s.n, m, s.S,
                           nh, (float)(s.n - (double)nh), mh, (float)(m - (double)mh),
                           (s.theta_s - s.theta_r) * s.alpha * s.n * m};
    }
    const long long N = c->g.N;
    std::vector<uint8_t> zone(N, 0);
    std::vector<double> Ks(N);
    for (long long p = 0; p < N; p++) {
        const int z = zone_of_cell ? zone_of_cell[p] : 0;
        if (z >= n_zones) return fail(RF_ERR_ARG, "zone_of_cell refers to an undefined zone");
        zone[p] = (uint8_t)z;
        Ks[p] = Ks_cell ? Ks_cell[p] : zones[z].Ks;
        if (c->flags_h[p] && !(Ks[p] > 0)) return fail(RF_ERR_ARG, "Ks_cell must be positive on active cells");
    }
    CUDA_TRY(cudaMemcpyAsync(c->soils, soils.data(), sizeof(DevSoil) * 256, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->zone, zone.data(), N, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->Ks, Ks.data(), sizeof(double) * N, cudaMemcpyHostToDevice, c->stream));
    if (rf_status st = sync(c)) return st;
    c->soils_set = true;
    c->has_state = false;   // closures depend on the soils: state must be set again
    c->closure_at_h = false;
    return RF_OK;
}

rf_status rf_bc_set(rf_ctx *c, rf_face face, rf_bc_type type, const double *t, const double *v, int n)
{
    if (!c || face < RF_XMIN || face > RF_ZMAX) return fail(RF_ERR_ARG, "bad face");
    if (type < RF_BC_ZERO_FLUX || type > RF_BC_SEEPAGE) return fail(RF_ERR_ARG, "bad boundary type");
    if (type == RF_BC_FREE_DRAINAGE && face != RF_ZMIN) return fail(RF_ERR_ARG, "free drainage is a bottom (ZMIN) condition");
    if ((type == RF_BC_DIRICHLET || type == RF_BC_FLUX) && (n < 1 || !v))
        return fail(RF_ERR_ARG, "Dirichlet and flux conditions need a value series");
    if (n > 1 && !t) return fail(RF_ERR_ARG, "a series of more than one value needs breakpoints");
    BcSeries b;
    b.type = type;
    if (v && n > 0) {
        for (int i = 0; i < n; i++) {
            b.t.push_back(t ? t[i] : 0.0);
            b.v.push_back(v[i]);
            if (!std::isfinite(v[i]) || !std::isfinite(b.t.back())) return fail(RF_ERR_ARG, "non-finite series");
            if (i > 0 && !(b.t[i] > b.t[i - 1])) return fail(RF_ERR_ARG, "breakpoints must increase strictly");
        }
    }
    c->bc[face] = b;
    return RF_OK;
}

static rf_status state_set_common(rf_ctx *c, double t)
{
    NvtxRange range("rf_state_set");
    c->t = t;
    c->dt_nom = std::min(c->prm.dt0, c->prm.dt_max);
    c->easy = 0;
    c->steps = 0;
    c->dt_prev = 0.0;           // the first step after a state is set is backward Euler
    c->err_last = c->err_max = 0.0;
    run_closure(c, c->h, nullptr, c->theta_n, 0);
    // closure_at_h promises K[0], C and theta_k at h: theta_k too (the
    // modified Picard form reads theta*(h^k) on the first iteration)
    CUDA_TRY(cudaMemcpyAsync(c->theta_k, c->theta_n, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice, c->stream));
    c->closure_at_h = true;
    double st0 = 0.0;
    if (rf_status st = storage_of_theta_n(c, &st0)) return st;
    c->storage0 = st0;
    c->in_cum = c->out_cum = c->closure_cum = c->defect_cum = 0.0;
    c->has_state = true;
    return RF_OK;
}

rf_status rf_state_set(rf_ctx *c, const double *h, double t)
{
    if (!c || !h) return fail(RF_ERR_ARG, "null argument");
    if (!c->soils_set) return fail(RF_ERR_STATE, "call rf_soil_set before rf_state_set");
    if (!std::isfinite(t)) return fail(RF_ERR_ARG, "non-finite time");
    // copied straight from the caller's buffer (a DMA when it is pinned) into
    // scratch, checked on the device, and committed only when every active
    // head is finite (the state is unchanged otherwise)
    CUDA_TRY(cudaMemcpyAsync(c->x, h, sizeof(double) * c->g.N, cudaMemcpyHostToDevice, c->stream));
    launch_state_check_commit(c->stream, c->nblk, c->g, c->flags, c->x, c->h, c->partials, c->ticket, c->res);
    CUDA_TRY(cudaMemcpyAsync(c->res_h, c->res, sizeof(StepResults), cudaMemcpyDeviceToHost, c->stream));
    if (rf_status st = sync(c)) return st;          // the host buffer is not read after this
    if (c->res_h->nonfinite) return fail(RF_ERR_ARG, "non-finite head on an active cell");
    return state_set_common(c, t);
}

rf_status rf_state_set_device(rf_ctx *c, const double *d_h, double t)
{
    if (!c || !d_h) return fail(RF_ERR_ARG, "null argument");
    if (!c->soils_set) return fail(RF_ERR_STATE, "call rf_soil_set before rf_state_set_device");
    CUDA_TRY(cudaMemcpyAsync(c->h, d_h, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice, c->stream));
    return state_set_common(c, t);
}

rf_status rf_state_get(rf_ctx *c, double *h, rf_state_meta *meta)
{
    if (!c) return fail(RF_ERR_ARG, "null context");
    if (h) {
        CUDA_TRY(cudaMemcpyAsync(h, c->h, sizeof(double) * c->g.N, cudaMemcpyDeviceToHost, c->stream));
        if (rf_status st = sync(c)) return st;
    }
    if (meta) {
        meta->t = c->t;
        meta->dt_nom = c->dt_nom;
        meta->easy = c->easy;
        meta->n_active = c->n_active;
        meta->steps = c->steps;
    }
    return RF_OK;
}

rf_status rf_state_get_device(rf_ctx *c, double *d_h)
{
    if (!c || !d_h) return fail(RF_ERR_ARG, "null argument");
    CUDA_TRY(cudaMemcpyAsync(d_h, c->h, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice, c->stream));
    return sync(c);
}

rf_status rf_state_meta_set(rf_ctx *c, const rf_state_meta *meta, const double *mass7)
{
    if (!c || !meta) return fail(RF_ERR_ARG, "null argument");
    if (!c->has_state) return fail(RF_ERR_STATE, "set the state first");
    c->t = meta->t;
    c->dt_nom = meta->dt_nom;
    c->easy = meta->easy;
    c->steps = meta->steps;
    if (mass7) {
        c->storage0 = mass7[0];
        c->in_cum = mass7[2];
        c->out_cum = mass7[3];
        c->closure_cum = mass7[4];
        c->defect_cum = mass7[6];
    }
    return RF_OK;
}

rf_status rf_step(rf_ctx *c, rf_step_info *out)
{
    NvtxRange range("rf_step");
    if (!c) return fail(RF_ERR_ARG, "null context");
    return step_any(c, INFINITY, out);
}

rf_status rf_run(rf_ctx *c, double t_end, rf_run_stats *stats, rf_step_info *log, int log_cap)
{
    NvtxRange range("rf_run");
    if (!c) return fail(RF_ERR_ARG, "null context");
    if (!std::isfinite(t_end)) return fail(RF_ERR_ARG, "non-finite t_end");
    rf_run_stats s{};
    rf_status st = RF_OK;
    while (c->t < t_end - t_tol(t_end)) {
        rf_step_info info{};
        st = step_any(c, t_end, &info);
        if (st) break;
        if (log && s.steps < log_cap) log[s.steps] = info;
        s.steps++;
        s.picard_iters += info.picard_iters;
        s.cg_iters += info.cg_iters;
        s.rejected += info.rejected;
    }
    if (stats) *stats = s;
    return st;
}

rf_status rf_mass_balance(rf_ctx *c, rf_mass_balance_t *out)
{
    if (!c || !out) return fail(RF_ERR_ARG, "null argument");
    if (!c->has_state) return fail(RF_ERR_STATE, "no state");
    double st = 0.0;
    if (rf_status s = storage_of_theta_n(c, &st)) return s;
    out->storage0 = c->storage0;
    out->storage = st;
    out->inflow_cum = c->in_cum;
    out->outflow_cum = c->out_cum;
    out->closure_abs = std::fabs(c->closure_cum);
    out->closure_rel = out->closure_abs / (c->storage0 + c->in_cum + c->out_cum);
    out->nonlinear_defect_cum = c->defect_cum;
    return RF_OK;
}

rf_status rf_assemble(rf_ctx *c, const double *d_hk, const double *d_hn, double dt, double t, double *d_K,
                      double *d_theta, double *d_c, double *d_b, double *d_diag)
{
    if (!c || !d_hk || !d_hn || !(dt > 0)) return fail(RF_ERR_ARG, "bad argument");
    if (!c->soils_set) return fail(RF_ERR_STATE, "soils not set");
    const double t_save = c->t;
    c->t = t;
    fill_step_params(c, dt);
    c->t = t_save;
    CUDA_TRY(cudaMemcpyAsync(c->sp, c->sp_h, sizeof(StepParams), cudaMemcpyHostToDevice, c->stream));
    // theta*(h^n) into theta_n's scratch twin, then closures at h^k
    run_closure(c, d_hn, nullptr, c->theta_n, 0);
    run_closure(c, d_hk, nullptr, c->theta_k, 0);
    run_assemble(c, d_hk, d_hn, c->theta_k, c->theta_n);
    c->closure_at_h = false;
    c->has_state = false;    // theta_n was overwritten: the state must be set again before stepping
    const size_t nb = sizeof(double) * c->g.N;
    if (d_K) CUDA_TRY(cudaMemcpyAsync(d_K, c->K[0], nb, cudaMemcpyDeviceToDevice, c->stream));
    if (d_theta) CUDA_TRY(cudaMemcpyAsync(d_theta, c->theta_k, nb, cudaMemcpyDeviceToDevice, c->stream));
    if (d_c) CUDA_TRY(cudaMemcpyAsync(d_c, c->c, nb, cudaMemcpyDeviceToDevice, c->stream));
    if (d_b) CUDA_TRY(cudaMemcpyAsync(d_b, c->b, nb, cudaMemcpyDeviceToDevice, c->stream));
    if (d_diag) CUDA_TRY(cudaMemcpyAsync(d_diag, c->diag, nb, cudaMemcpyDeviceToDevice, c->stream));
    return sync(c);
}

rf_status rf_apply(rf_ctx *c, const double *d_x, double *d_y)
{
    if (!c || !d_x || !d_y) return fail(RF_ERR_ARG, "null argument");
    launch_apply64(c->stream, c->nblk, c->g, c->flags, d_x, d_y, c->Tx, c->Ty, c->Tz, c->diag);
    return sync(c);
}

rf_status rf_solve(rf_ctx *c, double *d_x, int *iters)
{
    if (!c || !d_x) return fail(RF_ERR_ARG, "null argument");
    int it = 0;
    CUDA_TRY(cudaMemcpyAsync(c->hk, d_x, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice, c->stream));
    rf_status st = solve_system(c, &it);
    if (iters) *iters = it;
    if (st) return st;
    CUDA_TRY(cudaMemcpyAsync(d_x, c->x, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice, c->stream));
    c->has_state = false;   // hk was used as scratch
    return sync(c);
}

static bool ws_scales_ok(const rf_ws_scales *sc)
{
    return sc && sc->h_scale > 0 && std::isfinite(sc->lnK_mean) && sc->lnK_std > 0 && sc->q_scale > 0 &&
           sc->t_scale > 0 && std::isfinite(sc->out_scale) && std::isfinite(sc->h_scale) &&
           std::isfinite(sc->lnK_std) && std::isfinite(sc->q_scale) && std::isfinite(sc->t_scale);
}

static nn::WsScales ws_scales_of(const rf_ws_scales *sc)
{
    return nn::WsScales{sc->h_scale, sc->lnK_mean, sc->lnK_std, sc->q_scale, sc->t_scale, sc->out_scale};
}

rf_status rf_ws_features(rf_ctx *c, const rf_ws_scales *sc, const double *d_h, double t, double dt, float *d_x)
{
    if (!c || !d_x || !ws_scales_ok(sc) || !(dt > 0) || !std::isfinite(t)) return fail(RF_ERR_ARG, "bad argument");
    if ((reinterpret_cast<uintptr_t>(d_x) & 15u) != 0) return fail(RF_ERR_ARG, "d_x must be 16-byte aligned");
    if (!c->soils_set || (!d_h && !c->has_state)) return fail(RF_ERR_STATE, "set soils and state first");
    const nn::WsScales s = ws_scales_of(sc);
    float q_feat, dt_feat;
    ws_scalar_features(c, s, t, dt, q_feat, dt_feat);
    nn::ws_features_f32(c->stream, c->g, c->flags, d_h ? d_h : c->h, c->Ks, s, q_feat, dt_feat, d_x);
    CUDA_TRY(cudaGetLastError());
    return RF_OK;
}

rf_status rf_ws_target(rf_ctx *c, const rf_ws_scales *sc, const double *d_h_old, double dt, float *d_target,
                       float *d_mask)
{
    if (!c || !d_h_old || !d_target || !ws_scales_ok(sc) || !(dt > 0) || !(sc->out_scale != 0))
        return fail(RF_ERR_ARG, "bad argument");
    if (!c->has_state) return fail(RF_ERR_STATE, "no state");
    nn::ws_target(c->stream, c->g, c->flags, c->h, d_h_old, 1.0 / (sc->out_scale * dt), d_target, d_mask);
    CUDA_TRY(cudaGetLastError());
    return RF_OK;
}

rf_status rf_ws_attach(rf_ctx *c, rf_nn *net, const rf_ws_scales *sc)
{
    if (!c) return fail(RF_ERR_ARG, "ctx is NULL");
    if (net && !ws_scales_ok(sc)) return fail(RF_ERR_ARG, "invalid warm-start scales");
    c->ws_net = net;
    if (net) c->ws_sc = ws_scales_of(sc);
    c->ws_guesses = 0;
    c->ws_fallbacks = 0;
    return RF_OK;
}

rf_status rf_ws_get_stats(rf_ctx *c, rf_ws_stats *out)
{
    if (!c || !out) return fail(RF_ERR_ARG, "NULL argument");
    out->guesses = c->ws_guesses;
    out->fallbacks = c->ws_fallbacks;
    return RF_OK;
}

rf_status rf_apply_inner(rf_ctx *c, const float *d_z, const float *d_pold, float beta, float *d_p, float *d_q,
                         double *pq)
{
    if (!c || !d_z || !d_p || !d_q || (beta != 0.0f && !d_pold) || !std::isfinite(beta))
        return fail(RF_ERR_ARG, "bad argument");
    const Grid &g = c->g;
    cudaStream_t s = c->stream;
    const size_t nb = sizeof(float) * g.N;
    // the kernel reads z and p_old from the context's arrays (the TMA maps
    // describe them) and writes p into the other p buffer
    CUDA_TRY(cudaMemcpyAsync(c->z32, d_z, nb, cudaMemcpyDeviceToDevice, s));
    if (beta != 0.0f) CUDA_TRY(cudaMemcpyAsync(c->p32[1], d_pold, nb, cudaMemcpyDeviceToDevice, s));
    CgScal &h = *c->sc_in_h;
    h = CgScal{};
    h.iter = beta != 0.0f ? 1 : 0;      // iteration 0: p = z
    h.beta = beta;
    h.rho = 1.0;
    h.max_it = 1;
    CUDA_TRY(cudaMemcpyAsync(c->sc_in, c->sc_in_h, sizeof(CgScal), cudaMemcpyHostToDevice, s));
    launch_cg32_spmv(s, c->nblk, g, c->z32, c->p32[1], c->p32[0], c->q32, c->K32, c->cb32, c->partials, c->ticket,
                     c->sc_in, c->tma_ok ? &c->tma : nullptr, c->dev_fault);
    CUDA_TRY(cudaMemcpyAsync(d_p, c->p32[0], nb, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d_q, c->q32, nb, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->sc_in_h, c->sc_in, sizeof(CgScal), cudaMemcpyDeviceToHost, s));
    RF_TRY(sync(c));
    if (pq) *pq = c->sc_in_h->pq;
    return RF_OK;
}

rf_status rf_set_wait_limit(rf_ctx *c, int polls)
{
    if (!c) return fail(RF_ERR_ARG, "null context");
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->wait_polls = polls;
    c->g.wait_tries = polls;
    destroy_graphs(c);        // the grid (and its limit) is baked into the graphs
    return RF_OK;
}

unsigned long long rf_launch_count(rf_ctx *c)
{
    if (!c) return 0ULL;
    if (cudaMemcpyAsync(c->ctr_h, c->ctr, 2 * KK_COUNT * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return 0ULL;
    unsigned long long s = 0;
    for (int k = 0; k < KK_COUNT; k++) s += c->ctr_h[2 * k];
    return s;
}

int rf_launch_counts(rf_ctx *c, unsigned long long *out, int cap)
{
    if (!c || !out) return 0;
    if (cudaMemcpyAsync(c->ctr_h, c->ctr, 2 * KK_COUNT * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return 0;
    const int n = std::min(cap, 2 * (int)KK_COUNT);
    for (int i = 0; i < n; i++) out[i] = c->ctr_h[i];
    return n;
}

rf_status rf_profile_kernel(rf_ctx *c, int kind, int reps, double *avg_ms, double *bytes_per_launch)
{
    if (!c || reps < 1 || kind < RF_K_CLOSURE || kind > RF_K_CG32_UPDATE) return fail(RF_ERR_ARG, "bad argument");
    if (!c->has_state) return fail(RF_ERR_STATE, "set the state first");
    NvtxRange range("rf_profile_kernel");   // profilers can keep to these launches (ncu --nvtx-include)
    // algorithmic bytes per active cell (reads + writes, each array once)
    static const double per_cell[] = {50.0, 117.0, 65.0, 64.0, 65.0, 24.0, 32.0};
    static const bool reads_flags[] = {true, true, true, false, true, false, false};
    const Grid &g = c->g;
    const int nb = c->nblk;
    cudaStream_t s = c->stream;
    const CondSet none{0, 0};
    // the system at the current state
    fill_step_params(c, c->dt_nom);
    CUDA_TRY(cudaMemcpyAsync(c->sp, c->sp_h, sizeof(StepParams), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->hk, c->h, sizeof(double) * g.N, cudaMemcpyDeviceToDevice, s));
    run_closure(c, c->hk, nullptr, c->theta_k, 0);
    run_assemble(c, c->hk, c->h, c->theta_k, c->theta_n);
    c->closure_at_h = false;
    // the timed solves start from x0 = 0 (r0 = b, never zero) with a zero
    // tolerance and restart every 8 launches, so every timed launch does its
    // full work on values that stay meaningful whatever the state
    auto restart = [&]() -> rf_status {
        CUDA_TRY(cudaMemsetAsync(c->q, 0, sizeof(double) * g.N, s));
        if (kind == RF_K_CG64_SPMV || kind == RF_K_CG64_UPDATE)
            launch_cg64_init(s, nb, g, c->flags, c->q, c->x, c->b, c->Tx, c->Ty, c->Tz, c->diag, c->dinv, c->r, c->z,
                             0.0, 1 << 30, c->partials, c->ticket, c->sc, nullptr, none);
        if (kind >= RF_K_RESID64) {
            launch_mixed_start(s, nb, g, c->q, c->x, c->sc, c->sc_in, nullptr, none);
            launch_resid64(s, nb, g, c->flags, c->x, c->b, c->Tx, c->Ty, c->Tz, c->diag, c->dinv32, c->r32, c->z32,
                           c->d32, 0.0, 1e-30, 1 << 30, 1 << 30, c->partials, c->ticket, c->sc, c->sc_in, none, none);
        }
        // one untimed iteration, so the timed ones read the previous direction
        if (kind == RF_K_CG64_SPMV || kind == RF_K_CG64_UPDATE) {
            launch_cg64_spmv(s, nb, g, c->flags, c->z, c->p[1], c->p[0], c->q, c->Tx, c->Ty, c->Tz, c->diag,
                             c->partials, c->ticket, c->sc);
            launch_cg64_update(s, nb, g, c->x, c->r, c->z, c->p[0], c->q, c->dinv, c->partials, c->ticket, c->sc,
                               none);
        } else if (kind == RF_K_CG32_SPMV || kind == RF_K_CG32_UPDATE) {
            launch_cg32_spmv(s, nb, g, c->z32, c->p32[1], c->p32[0], c->q32, c->K32, c->cb32, c->partials, c->ticket,
                             c->sc_in, c->tma_ok ? &c->tma : nullptr, c->dev_fault);
            launch_cg32_update(s, nb, g, c->d32, c->r32, c->z32, c->p32[0], c->q32, c->dinv32, c->partials,
                               c->ticket, c->sc_in, none);
        }
        return RF_OK;
    };
    auto undone = [&]() {
        cudaMemsetAsync(&c->sc->done, 0, sizeof(int), s);
        cudaMemsetAsync(&c->sc_in->done, 0, sizeof(int), s);
    };
    std::vector<cudaEvent_t> ev(2 * reps);
    for (auto &e : ev) CUDA_TRY(cudaEventCreate(&e));
    for (int i = 0; i < reps; i++) {
        if (i % 8 == 0) RF_TRY(restart());
        double *pin = c->p[i & 1], *pout = c->p[(i + 1) & 1];
        float *qin = c->p32[i & 1], *qout = c->p32[(i + 1) & 1];
        // every timed launch does its full work: the solve is never marked
        // finished before it
        undone();
        auto timed = [&](auto &&launch) {
            undone();
            cudaEventRecord(ev[2 * i], s);
            launch();
            cudaEventRecord(ev[2 * i + 1], s);
        };
        switch (kind) {
        case RF_K_CLOSURE:
            timed([&] { launch_closure(s, nb, g, c->soils, c->zone, c->Ks, c->flags, c->hk, c->h, c->theta_k, c->K[1],
                                       c->Can, c->partials, c->ticket, c->res); });
            break;
        case RF_K_ASSEMBLE:
            timed([&] { run_assemble(c, c->hk, c->h, c->theta_k, c->theta_n); });
            break;
        case RF_K_CG64_SPMV:
        case RF_K_CG64_UPDATE:
            if (kind == RF_K_CG64_SPMV)
                timed([&] { launch_cg64_spmv(s, nb, g, c->flags, c->z, pin, pout, c->q, c->Tx, c->Ty, c->Tz, c->diag,
                                             c->partials, c->ticket, c->sc); });
            else
                launch_cg64_spmv(s, nb, g, c->flags, c->z, pin, pout, c->q, c->Tx, c->Ty, c->Tz, c->diag, c->partials,
                                 c->ticket, c->sc);
            if (kind == RF_K_CG64_UPDATE)
                timed([&] { launch_cg64_update(s, nb, g, c->x, c->r, c->z, pout, c->q, c->dinv, c->partials, c->ticket,
                                               c->sc, none); });
            else
                launch_cg64_update(s, nb, g, c->x, c->r, c->z, pout, c->q, c->dinv, c->partials, c->ticket, c->sc,
                                   none);
            break;
        case RF_K_RESID64:
            timed([&] { launch_resid64(s, nb, g, c->flags, c->x, c->b, c->Tx, c->Ty, c->Tz, c->diag, c->dinv32,
                                       c->r32, c->z32, c->d32, 0.0, 1e-30, 1 << 30, 1 << 30, c->partials, c->ticket,
                                       c->sc, c->sc_in, none, none); });
            break;
        default:
            if (kind == RF_K_CG32_SPMV)
                timed([&] { launch_cg32_spmv(s, nb, g, c->z32, qin, qout, c->q32, c->K32, c->cb32, c->partials,
                                             c->ticket, c->sc_in, c->tma_ok ? &c->tma : nullptr, c->dev_fault); });
            else
                launch_cg32_spmv(s, nb, g, c->z32, qin, qout, c->q32, c->K32, c->cb32, c->partials, c->ticket,
                                 c->sc_in, c->tma_ok ? &c->tma : nullptr, c->dev_fault);
            if (kind == RF_K_CG32_UPDATE)
                timed([&] { launch_cg32_update(s, nb, g, c->d32, c->r32, c->z32, qout, c->q32, c->dinv32, c->partials,
                                               c->ticket, c->sc_in, none); });
            else
                launch_cg32_update(s, nb, g, c->d32, c->r32, c->z32, qout, c->q32, c->dinv32, c->partials, c->ticket,
                                   c->sc_in, none);
            break;
        }
    }
    rf_status st = sync(c);
    double total = 0.0;
    for (int i = 0; st == RF_OK && i < reps; i++) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) != cudaSuccess) st = fail(RF_ERR_CUDA, "event timing");
        total += ms;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (st) return st;
    if (avg_ms) *avg_ms = total / reps;
    if (bytes_per_launch)
        *bytes_per_launch = per_cell[kind] * c->n_active + (reads_flags[kind] ? (double)g.N : 0.0);
    return RF_OK;
}

}  // extern "C"
