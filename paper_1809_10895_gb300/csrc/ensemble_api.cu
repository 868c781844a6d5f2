// ensemble_api.cu -- C ABI of the batched ensemble (rf_ens_*): packing of
// uneven instances, the persistent kernel captured in a CUDA graph, and the
// tuner that picks the tiling (cluster size, CTA size) and the schedule
// (queue order by measured work, instances run on whole clusters).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <queue>
#include <string>
#include <vector>

#include "ensemble.cuh"
#include "rf.h"

namespace rf {
// Validation of rf_solver_params shared with rf_mesh_create; sets the last error.
rf_status check_solver_params(const rf_solver_params *p);
}  // namespace rf

using namespace rf;

namespace {

rf_status efail(rf_status s, const std::string &m)
{
    set_last_error(m.c_str());
    return s;
}

#define ECUDA(x)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (x);                                                                             \
        if (e_ != cudaSuccess) return efail(RF_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

struct rf_ens {
    cudaStream_t stream = nullptr;
    rf_allocator alloc{};
    bool has_alloc = false;
    std::vector<void *> allocations;
    int n = 0, precision = 0, cluster = 1, threads = ENS_THREADS;
    long long ncells = 0;
    std::vector<int> order;            // queue position -> user index
    std::vector<int> pos;              // user index -> queue position
    std::vector<EnsDesc> desc0;        // initial descriptors (queue order)
    std::vector<double> h0;            // initial heads (packed, queue order)
    EnsDesc *D = nullptr;
    EnsBuffers B{};
    EnsParams P{};
    FFTables *tab = nullptr;
    unsigned long long *ctr = nullptr;
    double *t_end = nullptr, *t_end_h = nullptr;
    unsigned int *queue = nullptr;
    int *sched = nullptr;              // work queue: descriptor index | ENS_SCHED_WIDE
    std::vector<int> sched_h;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_cluster = 0, graph_threads = 0;

    void *dalloc(size_t bytes)
    {
        bytes = (bytes + 255) & ~size_t(255);
        void *ptr = nullptr;
        if (has_alloc) ptr = alloc.alloc(bytes, alloc.user);
        else if (cudaMalloc(&ptr, bytes) != cudaSuccess) ptr = nullptr;
        if (ptr) allocations.push_back(ptr);
        return ptr;
    }
    template <class T>
    bool get(T *&p, size_t n_)
    {
        p = static_cast<T *>(dalloc(sizeof(T) * (n_ ? n_ : 1)));
        return p != nullptr;
    }
};

namespace {

void destroy_graph(rf_ens *e)
{
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    e->exec = nullptr;
    e->graph = nullptr;
    e->graph_cluster = 0;
    e->graph_threads = 0;
}

// Schedule from an order of descriptor indices; the first n_wide run on
// whole clusters.
rf_status upload_schedule(rf_ens *e, const std::vector<int> &desc_order, int n_wide)
{
    e->sched_h.resize(e->n);
    for (int k = 0; k < e->n; k++) e->sched_h[k] = desc_order[k] | (k < n_wide ? ENS_SCHED_WIDE : 0);
    ECUDA(cudaMemcpyAsync(e->sched, e->sched_h.data(), sizeof(int) * e->n, cudaMemcpyHostToDevice, e->stream));
    ECUDA(cudaStreamSynchronize(e->stream));
    return RF_OK;
}

rf_status upload_initial(rf_ens *e)
{
    ECUDA(cudaMemcpyAsync(e->D, e->desc0.data(), sizeof(EnsDesc) * e->n, cudaMemcpyHostToDevice, e->stream));
    ECUDA(cudaMemcpyAsync(e->B.H[0], e->h0.data(), sizeof(double) * e->ncells, cudaMemcpyHostToDevice, e->stream));
    ECUDA(cudaStreamSynchronize(e->stream));
    return RF_OK;
}

// One graph: queue reset, then the persistent kernel.
rf_status build_graph(rf_ens *e)
{
    destroy_graph(e);
    const int ncl = ensemble_max_clusters(e->cluster, e->threads, e->precision);
    if (ncl < 1) return efail(RF_ERR_CUDA, "no cluster of that size fits on this device");
    cudaStream_t cap;
    ECUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (err == cudaSuccess) err = cudaMemsetAsync(e->queue, 0, sizeof(unsigned int), cap);
    if (err == cudaSuccess)
        err = launch_ensemble(cap, e->cluster, e->threads, ncl, e->precision, e->D, e->n, e->B, e->P, e->t_end,
                              e->queue, e->sched);
    cudaGraph_t g = nullptr;
    const cudaError_t err2 = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (err != cudaSuccess || err2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return efail(RF_ERR_CUDA, std::string("ensemble graph capture: ") +
                                      cudaGetErrorString(err != cudaSuccess ? err : err2));
    }
    e->graph = g;
    ECUDA(cudaGraphInstantiate(&e->exec, g, 0));
    e->graph_cluster = e->cluster;
    e->graph_threads = e->threads;
    return RF_OK;
}

// List-scheduling model of the persistent queue: `units` work units of
// `cluster` CTAs pop instances in `order`; the first n_wide run on a whole
// unit for wide_s[i]; the first other pop splits its unit into `cluster`
// single CTAs (the popping CTA runs that instance), and single CTAs run
// instances for solo_s[i].  Units that free at the same time pop single CTAs
// first.  Returns when the last instance ends.
double model_makespan(const double *wide_s, const double *solo_s, const int *order, int n, int n_wide, int units,
                      int cluster)
{
    // (free time, is a whole cluster) per unit, earliest first
    std::priority_queue<std::pair<double, int>, std::vector<std::pair<double, int>>,
                        std::greater<std::pair<double, int>>> q;
    for (int u = 0; u < units; u++) q.push({0.0, 1});
    double end = 0.0;
    int k = 0;
    while (!q.empty()) {
        auto [t, whole] = q.top();
        q.pop();
        if (k >= n) {
            end = std::max(end, t);
            continue;
        }
        const int d = order[k];
        if (whole && k < n_wide) {
            q.push({t + wide_s[d], 1});
        } else {
            if (whole)
                for (int r = 1; r < cluster; r++) q.push({t, 0});
            q.push({t + solo_s[d], 0});
        }
        k++;
    }
    return end;
}

}  // namespace

extern "C" {

rf_status rf_ens_create(const rf_ens_instance *inst, int n, const rf_solver_params *params, void *cuda_stream,
                        const rf_allocator *alloc, rf_ens **out)
{
    if (out) *out = nullptr;
    if (!inst || n < 1 || !out) return efail(RF_ERR_ARG, "rf_ens_create: need at least one instance");
    rf_solver_params prm;
    rf_default_params(&prm);
    if (params) prm = *params;
    if (rf_status st = check_solver_params(&prm)) return st;
    if (prm.picard_form != RF_PICARD_CHORD)
        return efail(RF_ERR_ARG, "rf_ens_create: the ensemble runs the classical (chord) Picard iteration only");
    if (prm.precond != RF_PRECOND_JACOBI && prm.precond != RF_PRECOND_ZLINE)
        return efail(RF_ERR_ARG, "rf_ens_create: the ensemble's PCG is Jacobi- or vertical-line-preconditioned only");
    if (prm.face_mean != RF_FACE_ARITHMETIC || prm.time_scheme != RF_TIME_BACKWARD_EULER ||
        prm.time_control != RF_TIME_EBATS || prm.grav[0] != 0.0 || prm.grav[1] != 0.0 || prm.grav[2] != 1.0)
        return efail(RF_ERR_ARG, "rf_ens_create: the ensemble runs the default scheme (arithmetic face mean, "
                                 "backward Euler under EBATS, z-up gravity) only");
    long long total = 0;
    for (int i = 0; i < n; i++) {
        const rf_ens_instance &a = inst[i];
        if (a.nx < 1 || a.ny < 1 || a.nz < 1 || !(a.dx > 0) || !(a.dy > 0) || !(a.dz > 0))
            return efail(RF_ERR_ARG, "rf_ens_create: bad grid in instance " + std::to_string(i));
        const rf_soil &s = a.soil;
        if ((s.model != RF_VG && s.model != RF_GARDNER) || !(s.theta_s > s.theta_r) || !(s.alpha > 0) ||
            !(s.Ks > 0) || !(s.S >= 0) || (s.model == RF_VG && !(s.n > 1.0)))
            return efail(RF_ERR_ARG, "rf_ens_create: bad soil in instance " + std::to_string(i));
        if (a.top_type != RF_BC_DIRICHLET && a.top_type != RF_BC_FLUX && a.top_type != RF_BC_ZERO_FLUX)
            return efail(RF_ERR_ARG, "rf_ens_create: top must be Dirichlet, flux or zero flux");
        if (a.bottom_type != RF_BC_FREE_DRAINAGE && a.bottom_type != RF_BC_DIRICHLET &&
            a.bottom_type != RF_BC_ZERO_FLUX)
            return efail(RF_ERR_ARG, "rf_ens_create: bottom must be free drainage, Dirichlet or zero flux");
        total += (long long)a.nx * a.ny * a.nz;
    }
    if (total > (1LL << 31) - 1) return efail(RF_ERR_ARG, "rf_ens_create: too many cells");

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return efail(RF_ERR_NO_DEVICE, "no CUDA device visible; this library has no CPU fallback");
    }
    int dev = 0;
    ECUDA(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    ECUDA(cudaGetDeviceProperties(&prop, dev));
    if (prop.major != 10 || prop.minor != 3)
        return efail(RF_ERR_NO_DEVICE, "this library is built for sm_103a (GB300) only");

    rf_ens *e = new rf_ens();
    e->stream = static_cast<cudaStream_t>(cuda_stream);
    if (alloc && alloc->alloc && alloc->free) { e->alloc = *alloc; e->has_alloc = true; }
    e->n = n;
    e->precision = prm.precision;
    e->ncells = total;
    // largest instances first in the work queue
    e->order.resize(n);
    std::iota(e->order.begin(), e->order.end(), 0);
    auto cells = [&](int i) { return (long long)inst[i].nx * inst[i].ny * inst[i].nz; };
    std::stable_sort(e->order.begin(), e->order.end(), [&](int a, int b) { return cells(a) > cells(b); });
    e->pos.resize(n);
    for (int k = 0; k < n; k++) e->pos[e->order[k]] = k;

    const long long N = total;
    bool ok = e->get(e->D, n) && e->get(e->tab, 1) && e->get(e->ctr, 2 * KK_COUNT) && e->get(e->t_end, 1) &&
              e->get(e->queue, 1) && e->get(e->sched, n);
    for (int b = 0; b < 3 && ok; b++) ok = e->get(e->B.H[b], N);
    for (int b = 0; b < 2 && ok; b++) ok = e->get(e->B.TH[b], N) && e->get(e->B.K[b], N) && e->get(e->B.p[b], N) &&
                                            e->get(e->B.p32[b], N);
    ok = ok && e->get(e->B.Can, N) && e->get(e->B.c, N) && e->get(e->B.b, N) && e->get(e->B.Tx, N) &&
         e->get(e->B.Ty, N) && e->get(e->B.Tz, N) && e->get(e->B.diag, N) && e->get(e->B.dinv, N) &&
         e->get(e->B.r, N) && e->get(e->B.z, N) && e->get(e->B.q, N) && e->get(e->B.K32, N) &&
         e->get(e->B.cb32, N) && e->get(e->B.dinv32, N) && e->get(e->B.r32, N) && e->get(e->B.z32, N) &&
         e->get(e->B.q32, N) && e->get(e->B.d32, N) && e->get(e->B.flags, N) && e->get(e->B.zone, N) &&
         e->get(e->B.Ks, N);
    if (ok && prm.precond == RF_PRECOND_ZLINE)
        ok = e->get(e->B.lt_inv, N) && e->get(e->B.lt_c, N) && e->get(e->B.lt_P, N) && e->get(e->B.lt_Q, N) &&
             e->get(e->B.lt_rs, N);
    if (!ok || cudaMallocHost(&e->t_end_h, sizeof(double)) != cudaSuccess) {
        rf_ens_destroy(e);
        return efail(RF_ERR_NOMEM, "rf_ens_create: allocation failed");
    }

    FFTables tab;
    make_ff_tables(&tab);
    std::vector<uint8_t> flags(N), zone(N, 0);
    std::vector<double> Ks(N);
    e->h0.assign(N, 0.0);
    e->desc0.resize(n);
    long long off = 0;
    for (int k = 0; k < n; k++) {
        const rf_ens_instance &a = inst[e->order[k]];
        EnsDesc d{};
        Grid &g = d.g;
        g.nx = a.nx; g.ny = a.ny; g.nz = a.nz;
        g.N = (long long)a.nx * a.ny * a.nz;
        g.sxy = (long long)a.nx * a.ny;
        g.V = a.dx * a.dy * a.dz;
        const double A[6] = {a.dy * a.dz, a.dy * a.dz, a.dx * a.dz, a.dx * a.dz, a.dx * a.dy, a.dx * a.dy};
        const double dd[6] = {a.dx, a.dx, a.dy, a.dy, a.dz, a.dz};
        for (int f = 0; f < 6; f++) {
            g.A[f] = A[f];
            g.w[f] = A[f] / dd[f];
            g.wb[f] = A[f] / (0.5 * dd[f]);
            g.hw[f] = 0.5 * (A[f] / dd[f]);
            g.gf[f] = f == F_ZMIN ? -1.0 : (f == F_ZMAX ? 1.0 : 0.0);
            g.hg[f] = 0.5 * A[f] * g.gf[f];
        }
        // closures in FP64 on the plain path, double-float inside the mixed one (AUTO)
        g.closure64 = (prm.closure_arith == RF_CLOSURE_FP64 ||
                       (prm.closure_arith == RF_CLOSURE_AUTO && prm.precision == RF_PREC_FP64)) ? 1 : 0;
        for (int ax = 0; ax < 3; ax++) g.w32[ax] = (float)(A[2 * ax] / dd[2 * ax]);
        g.fx = make_fastdiv((unsigned int)a.nx);
        g.fxy = make_fastdiv((unsigned int)g.sxy);
        g.tab = e->tab;
        g.ctr = e->ctr;
        const rf_soil &s = a.soil;
        const double m = s.model == RF_VG ? 1.0 - 1.0 / s.n : 0.0;
        const float nh = (float)s.n, mh = (float)m;
        d.soil = DevSoil{s.model, s.theta_r, s.theta_s, s.alpha, s.n, m, s.S, nh, (float)(s.n - (double)nh), mh,
                         (float)(m - (double)mh), (s.theta_s - s.theta_r) * s.alpha * s.n * m};
        for (int f = 0; f < 6; f++) { d.sp.bc_type[f] = BC_ZERO_FLUX; d.sp.bc_val[f] = 0.0; }
        d.sp.bc_type[F_ZMAX] = a.top_type;
        d.sp.bc_val[F_ZMAX] = a.top_value;
        d.sp.bc_type[F_ZMIN] = a.bottom_type;
        d.sp.bc_val[F_ZMIN] = a.bottom_value;
        d.sp.eps_chord = prm.eps_chord;
        d.off = off;
        d.t = 0.0;
        d.dt_nom = std::min(prm.dt0, prm.dt_max);
        d.status = ENS_NEW;
        e->desc0[k] = d;
        for (int kk = 0; kk < a.nz; kk++)
            for (int j = 0; j < a.ny; j++)
                for (int i = 0; i < a.nx; i++) {
                    const long long p = off + i + (long long)a.nx * (j + (long long)a.ny * kk);
                    uint8_t fl = FLAG_ACTIVE;
                    if (i == 0) fl |= 1u << F_XMIN;
                    if (i == a.nx - 1) fl |= 1u << F_XMAX;
                    if (j == 0) fl |= 1u << F_YMIN;
                    if (j == a.ny - 1) fl |= 1u << F_YMAX;
                    if (kk == 0) fl |= 1u << F_ZMIN;
                    if (kk == a.nz - 1) fl |= 1u << F_ZMAX;
                    flags[p] = fl;
                    Ks[p] = s.Ks;
                    e->h0[p] = a.h0;
                }
        off += g.N;
    }
    EnsParams &P = e->P;
    P.tol_picard = prm.tol_picard;
    P.tol_cg = prm.tol_cg;
    P.tol_inner = prm.tol_inner;
    P.dt_max = prm.dt_max;
    P.dt_min = prm.dt_min;
    P.f_grow = prm.f_grow;
    P.f_shrink = prm.f_shrink;
    P.eps_chord = prm.eps_chord;
    P.n_inc = prm.n_inc;
    P.n_small = prm.n_small;
    P.n_max = prm.n_max;
    P.cg_max_it = prm.cg_max_it;
    P.inner_max_it = prm.inner_max_it;
    P.outer_max_it = prm.outer_max_it;
    P.zline = prm.precond == RF_PRECOND_ZLINE;
    P.step_budget = 10000000;
    cudaError_t err = cudaMemcpyAsync(e->tab, &tab, sizeof(FFTables), cudaMemcpyHostToDevice, e->stream);
    if (err == cudaSuccess) err = cudaMemcpyAsync(e->B.flags, flags.data(), N, cudaMemcpyHostToDevice, e->stream);
    if (err == cudaSuccess) err = cudaMemcpyAsync(e->B.zone, zone.data(), N, cudaMemcpyHostToDevice, e->stream);
    if (err == cudaSuccess) err = cudaMemcpyAsync(e->B.Ks, Ks.data(), sizeof(double) * N, cudaMemcpyHostToDevice, e->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(e->ctr, 0, 2 * KK_COUNT * sizeof(unsigned long long), e->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
    if (err != cudaSuccess) {
        rf_ens_destroy(e);
        return efail(RF_ERR_CUDA, std::string("rf_ens_create: ") + cudaGetErrorString(err));
    }
    std::vector<int> size_order(n);
    std::iota(size_order.begin(), size_order.end(), 0);
    rf_status st = upload_initial(e);
    if (!st) st = upload_schedule(e, size_order, n);
    if (st) {
        rf_ens_destroy(e);
        return st;
    }
    *out = e;
    return RF_OK;
}

void rf_ens_destroy(rf_ens *e)
{
    if (!e) return;
    cudaStreamSynchronize(e->stream);
    destroy_graph(e);
    for (void *p : e->allocations) {
        if (e->has_alloc) e->alloc.free(p, e->alloc.user);
        else cudaFree(p);
    }
    if (e->t_end_h) cudaFreeHost(e->t_end_h);
    delete e;
}

rf_status rf_ens_set_tiling(rf_ens *e, int cluster, int threads)
{
    if (!e || (cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8))
        return efail(RF_ERR_ARG, "rf_ens_set_tiling: cluster must be 1, 2, 4 or 8");
    if (threads != 128 && threads != 256 && threads != 512)
        return efail(RF_ERR_ARG, "rf_ens_set_tiling: threads must be 128, 256 or 512");
    if (ensemble_max_clusters(cluster, threads, e->precision) < 1)
        return efail(RF_ERR_ARG, "rf_ens_set_tiling: clusters of that size do not fit on this device");
    e->cluster = cluster;
    e->threads = threads;
    return RF_OK;
}

rf_status rf_ens_set_schedule(rf_ens *e, const int *order, int n_wide)
{
    if (!e) return efail(RF_ERR_ARG, "null ensemble");
    std::vector<int> desc_order(e->n);
    if (order) {
        std::vector<char> seen(e->n, 0);
        for (int k = 0; k < e->n; k++) {
            const int i = order[k];
            if (i < 0 || i >= e->n || seen[i])
                return efail(RF_ERR_ARG, "rf_ens_set_schedule: order must be a permutation of the instances");
            seen[i] = 1;
            desc_order[k] = e->pos[i];
        }
    } else {
        std::iota(desc_order.begin(), desc_order.end(), 0);
    }
    return upload_schedule(e, desc_order, n_wide < 0 || n_wide > e->n ? e->n : n_wide);
}

rf_status rf_ens_run(rf_ens *e, double t_end)
{
    rf::NvtxRange range("rf_ens_run");
    if (!e || !std::isfinite(t_end)) return efail(RF_ERR_ARG, "rf_ens_run: bad argument");
    if (!e->exec || e->graph_cluster != e->cluster || e->graph_threads != e->threads)
        if (rf_status st = build_graph(e)) return st;
    *e->t_end_h = t_end;
    ECUDA(cudaMemcpyAsync(e->t_end, e->t_end_h, sizeof(double), cudaMemcpyHostToDevice, e->stream));
    ECUDA(cudaGraphLaunch(e->exec, e->stream));
    ECUDA(cudaStreamSynchronize(e->stream));
    ECUDA(cudaGetLastError());
    return RF_OK;
}

rf_status rf_ens_get(rf_ens *e, int i, double *h, rf_ens_stats *st)
{
    if (!e || i < 0 || i >= e->n) return efail(RF_ERR_ARG, "rf_ens_get: bad instance index");
    const int k = e->pos[i];
    EnsDesc d;
    ECUDA(cudaMemcpyAsync(&d, e->D + k, sizeof(EnsDesc), cudaMemcpyDeviceToHost, e->stream));
    ECUDA(cudaStreamSynchronize(e->stream));
    if (h) {
        const int hb = d.status == ENS_NEW ? 0 : d.hbuf;
        ECUDA(cudaMemcpyAsync(h, e->B.H[hb] + d.off, sizeof(double) * d.g.N, cudaMemcpyDeviceToHost, e->stream));
        ECUDA(cudaStreamSynchronize(e->stream));
    }
    if (st) {
        st->t = d.t;
        st->dt_nom = d.dt_nom;
        st->steps = d.steps;
        st->picard_iters = d.picard;
        st->cg_iters = d.cg;
        st->rejected = d.rejected;
        st->status = d.status == ENS_DT_MIN ? RF_ERR_DT_MIN : (d.status == ENS_BUDGET ? RF_ERR_DEVICE_TIMEOUT : RF_OK);
        st->cells = d.g.N;
        st->storage0 = d.storage0;
        st->inflow_cum = d.in_cum;
        st->outflow_cum = d.out_cum;
        st->closure_abs = std::fabs(d.closure_cum);
        st->nonlinear_defect_cum = d.defect_cum;
        st->busy_s = 1e-9 * (double)d.busy_ns;
        st->ctas = d.ctas;
    }
    return RF_OK;
}

rf_status rf_ens_reset(rf_ens *e)
{
    if (!e) return efail(RF_ERR_ARG, "null ensemble");
    return upload_initial(e);
}

rf_status rf_ens_tune(rf_ens *e, double t_probe, int *best_cluster, int *best_threads, int *best_wide,
                      double *best_ms)
{
    if (!e || !(t_probe > 0)) return efail(RF_ERR_ARG, "rf_ens_tune: bad argument");
    const int n = e->n;
    // timing events, released on every return path
    struct Events {
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events()
        {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    ECUDA(cudaEventCreate(&ev.a));
    ECUDA(cudaEventCreate(&ev.b));
    cudaEvent_t a = ev.a, b = ev.b;
    std::vector<EnsDesc> dh(n);
    // one timed run from the initial state; busy[k] = seconds descriptor k held its unit
    auto probe = [&](int c, int th, const std::vector<int> &ord, int n_wide, float &ms,
                     std::vector<double> *busy) -> rf_status {
        e->cluster = c;
        e->threads = th;
        if (rf_status st = upload_initial(e)) return st;
        if (rf_status st = upload_schedule(e, ord, n_wide)) return st;
        if (rf_status st = build_graph(e)) return st;
        *e->t_end_h = t_probe;
        ECUDA(cudaMemcpyAsync(e->t_end, e->t_end_h, sizeof(double), cudaMemcpyHostToDevice, e->stream));
        ECUDA(cudaEventRecord(a, e->stream));
        ECUDA(cudaGraphLaunch(e->exec, e->stream));
        ECUDA(cudaEventRecord(b, e->stream));
        ECUDA(cudaEventSynchronize(b));
        ECUDA(cudaEventElapsedTime(&ms, a, b));
        if (busy) {
            ECUDA(cudaMemcpyAsync(dh.data(), e->D, sizeof(EnsDesc) * n, cudaMemcpyDeviceToHost, e->stream));
            ECUDA(cudaStreamSynchronize(e->stream));
            busy->resize(n);
            for (int k = 0; k < n; k++) (*busy)[k] = 1e-9 * (double)dh[k].busy_ns;
        }
        return RF_OK;
    };
    struct Cand {
        int c, th, wide;
        double t;
        std::vector<int> order;
    };
    std::vector<int> size_order(n);
    std::iota(size_order.begin(), size_order.end(), 0);
    Cand best{0, 0, n, INFINITY, size_order};
    // 1. every tiling with every instance on a whole unit, largest first:
    // a timed run, and each instance's time at that width
    const int ths[2] = {512, 256}, cls[4] = {1, 2, 4, 8};
    std::vector<double> busy[2][4];
    int ncl[2][4] = {};
    for (int ti = 0; ti < 2; ti++)
        for (int ci = 0; ci < 4; ci++) {
            ncl[ti][ci] = ensemble_max_clusters(cls[ci], ths[ti], e->precision);
            if (ncl[ti][ci] < 1) continue;
            float ms = 0.0f;
            if (rf_status st = probe(cls[ci], ths[ti], size_order, n, ms, &busy[ti][ci])) return st;
            if (ms < best.t) best = Cand{cls[ci], ths[ti], n, ms, size_order};
        }
    if (!best.c) return efail(RF_ERR_CUDA, "rf_ens_tune: no tiling fits");
    // 2. list-scheduling model of the persistent kernel: ncl clusters pop the
    // queue (heaviest first at that width), each instance holding its
    // cluster for its measured time.  Every instance stays wide: a split
    // schedule (the lighter instances on single CTAs) is left to callers
    // that know the per-instance costs over their whole window -- from a
    // short probe it is unsafe, since an instance light early in the window
    // can turn heavy later and become the critical path on one CTA.  The
    // model's n_wide loop is kept general for that use.
    std::vector<Cand> preds;
    for (int ti = 0; ti < 2; ti++) {
        if (ncl[ti][0] < 1) continue;
        const std::vector<double> &solo = busy[ti][0];
        for (int ci = 1; ci < 4; ci++) {
            if (ncl[ti][ci] < 1) continue;
            const std::vector<double> &wide = busy[ti][ci];
            const int c = cls[ci], units = ncl[ti][ci];
            std::vector<int> lpt = size_order;
            std::stable_sort(lpt.begin(), lpt.end(), [&](int x, int y) { return wide[x] > wide[y]; });
            for (int w = n; w <= n; w++)
                preds.push_back(Cand{c, ths[ti], w,
                                     model_makespan(wide.data(), solo.data(), lpt.data(), n, w, units, c), lpt});
        }
    }
    std::stable_sort(preds.begin(), preds.end(), [](const Cand &x, const Cand &y) { return x.t < y.t; });
    // 3. time the three best predictions; keep the fastest measured run
    for (size_t i = 0; i < preds.size() && i < 3; i++) {
        float ms = 0.0f;
        if (rf_status st = probe(preds[i].c, preds[i].th, preds[i].order, preds[i].wide, ms, nullptr)) return st;
        if (ms < best.t) best = Cand{preds[i].c, preds[i].th, preds[i].wide, ms, preds[i].order};
    }
    e->cluster = best.c;
    e->threads = best.th;
    if (rf_status st = upload_schedule(e, best.order, best.wide)) return st;
    if (rf_status st = upload_initial(e)) return st;
    if (best_cluster) *best_cluster = best.c;
    if (best_threads) *best_threads = best.th;
    if (best_wide) *best_wide = best.wide;
    if (best_ms) *best_ms = best.t;
    return RF_OK;
}

rf_status rf_ens_model_makespan(const double *wide_s, const double *solo_s, const int *order, int n, int n_wide,
                                int units, int cluster, double *makespan)
{
    if (!wide_s || !order || !makespan || n < 1 || units < 1 || cluster < 1 || n_wide < 0)
        return efail(RF_ERR_ARG, "rf_ens_model_makespan: bad argument");
    if (n_wide < n && !solo_s) return efail(RF_ERR_ARG, "rf_ens_model_makespan: split schedules need solo_s");
    std::vector<char> seen(n, 0);
    for (int k = 0; k < n; k++) {
        if (order[k] < 0 || order[k] >= n || seen[order[k]])
            return efail(RF_ERR_ARG, "rf_ens_model_makespan: order must be a permutation");
        seen[order[k]] = 1;
    }
    *makespan = model_makespan(wide_s, solo_s ? solo_s : wide_s, order, n, n_wide > n ? n : n_wide, units, cluster);
    return RF_OK;
}

}  // extern "C"
