/*
 * Host side of the bmpc C ABI (include/bmpc.h): tree validation, device layout,
 * packing of problem data into one staging buffer, one host-to-device copy per
 * upload, the persistent solver launch (optionally captured into a CUDA graph)
 * and unpacking of the results.  The library allocates no device memory: all
 * device regions are carved out of the two caller-owned arenas.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <thread>
#include <vector>

#include "../../include/bmpc.h"
#include "bmpc_layout.h"
#include "../../include/bmpc_mlp.h"

namespace bmpc {
cudaError_t launch_solve(const KernelArgs &args, int model, int grid, int block, size_t smem, cudaStream_t stream);
size_t solve_smem(int model, int tab_ints, int max_paths, int block, int *stg_ld);
cudaError_t prepare_solve(int model, size_t smem);
cudaError_t launch_order(const ProbRec *recs, const Stats *stats, int32_t *order, int cnt, cudaStream_t stream);
cudaError_t launch_flat(int which, const FlatArgs &a, int n_problems, cudaStream_t stream);
cudaError_t launch_sincos(const float *a, float *sn, float *cs, int n, cudaStream_t stream);
cudaError_t launch_eig(float *S, int n, int count, cudaStream_t stream);
cudaError_t launch_dynhess(int model, const float *params, float dt, const float *x, const float *u, const float *mu,
                           float *H, int count, cudaStream_t stream);
cudaError_t launch_fma(float *out, int blocks, int iters, cudaStream_t stream);
int max_block_threads();
cudaError_t occupancy(int model, int block, size_t smem, int *blocks_per_sm, const KOpts &o);
cudaError_t launch_scatter_warm(const WarmArgs &a, cudaStream_t stream);
cudaError_t launch_shift_warm(const WarmArgs &a, int model, cudaStream_t stream);
cudaError_t launch_glue(int which, const GlueArgs &a, int n_problems, cudaStream_t stream, int model);
}  // namespace bmpc

using namespace bmpc;

static_assert(sizeof(Stats) == sizeof(bmpc_stats), "device statistics must match the public struct");

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int n_con(const bmpc_tree_desc &d) { return 2 * NU * (d.box_on ? 1 : 0) + d.n_obs + 2 * (d.lane_on ? 1 : 0); }

/* Tree checks: level order, children contiguous, model/size consistency. */
int validate(const bmpc_tree_desc &d, std::vector<int> *stage_out) {
    if (d.num_nodes < 2 || !d.parent) return BMPC_ERR_INVALID;
    if (d.nu != NU) return BMPC_ERR_INVALID;
    if (d.model == 0 && d.nx != 4) return BMPC_ERR_INVALID;
    if (d.model == 1 && d.nx != 6) return BMPC_ERR_INVALID;
    if ((d.model == 2 || d.model == 3) && d.nx != 4) return BMPC_ERR_INVALID;
    if (d.model < 0 || d.model >= NUM_MODELS) return BMPC_ERR_INVALID;
    if (d.n_obs < 0 || d.n_obs > MAX_OBS) return BMPC_ERR_INVALID;
    if (!(d.dt > 0.f) || !std::isfinite(d.dt)) return BMPC_ERR_INVALID;
    if (d.model != 2 && !(d.params[9] >= 1.f && d.params[9] <= 64.f)) return BMPC_ERR_INVALID;
    if (d.edge_dynamics != 0 && (d.edge_dynamics != 1 || d.model != 2)) return BMPC_ERR_INVALID;
    const int n = d.num_nodes;
    std::vector<int> stage(n, 0);
    if (d.parent[0] != -1) return BMPC_ERR_INVALID;
    for (int i = 1; i < n; ++i) {
        const int p = d.parent[i];
        if (p < 0 || p >= i) return BMPC_ERR_INVALID;
        if (i >= 2 && p < d.parent[i - 1]) return BMPC_ERR_INVALID;   /* children contiguous */
        stage[i] = stage[p] + 1;
        if (stage[i] < stage[i - 1]) return BMPC_ERR_INVALID;          /* level order */
    }
    if (stage_out) *stage_out = std::move(stage);
    return BMPC_OK;
}

/* Segment order of the scan sweeps (layout in bmpc_layout.h): the node at every position, the
 * position of its segment's end, the first position of every wave and the longest segment (in
 * nodes) of every wave.  Nodes are in level order with contiguous children. */
struct Segments {
    std::vector<int32_t> fnode, fend, wstart, wmax;
};
void segments(int n, const int32_t *parent, Segments &S) {
    std::vector<int> nch(n, 0), fch(n, 0), stage(n, 0), end(n, 0), wave(n, 0), size(n, 0);
    for (int i = 1; i < n; ++i) {
        const int p = parent[i];
        if (nch[p] == 0) fch[p] = i;
        nch[p]++;
        stage[i] = stage[p] + 1;
    }
    for (int i = n - 1; i >= 0; --i) end[i] = nch[i] == 1 ? end[fch[i]] : i;
    int W = 0;
    for (int i = n - 1; i >= 0; --i) {
        size[end[i]]++;
        if (nch[i] == 1) continue;
        int w = 0;
        for (int c = fch[i]; c < fch[i] + nch[i]; ++c) w = std::max(w, wave[end[c]] + 1);
        wave[i] = w;
        W = std::max(W, w + 1);
    }
    std::vector<int> idx(n), pos(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        const int ea = end[a], eb = end[b];
        if (wave[ea] != wave[eb]) return wave[ea] < wave[eb];
        if (ea != eb) return ea < eb;
        return stage[a] < stage[b];
    });
    S.fnode.assign(idx.begin(), idx.end());
    for (int f = 0; f < n; ++f) pos[idx[f]] = f;
    S.fend.resize(n);
    for (int f = 0; f < n; ++f) S.fend[f] = pos[end[idx[f]]];
    S.wstart.assign(W + 1, 0);
    S.wmax.assign(W, 0);
    for (int i = 0; i < n; ++i) {
        S.wstart[wave[end[i]] + 1]++;
        if (end[i] == i) S.wmax[wave[i]] = std::max(S.wmax[wave[i]], size[i]);
    }
    for (int w = 0; w < W; ++w) S.wstart[w + 1] += S.wstart[w];
}

struct Layout {
    size_t recs, order, queue, ints, in, warm, out, stats, raw, data_total;   /* byte offsets in the data arena */
    size_t ints_n, in_n, warm_n, out_n, scr_n, raw_n;                         /* element counts */
    int64_t T_n, T_nx, T_nc, T_obs;                                          /* node-major flat totals */
    size_t staging;
};

}  // namespace

struct bmpc_batch {
    int n = 0;
    std::vector<ProbRec> recs;
    std::vector<int32_t> order;
    std::vector<int> nodes;
    std::vector<int32_t> parents;        /* all trees' parent arrays, concatenated */
    int model_begin[NUM_MODELS + 1] = {};  /* order[model_begin[m] .. model_begin[m+1]) has model m */
    int tab_ints[NUM_MODELS] = {};         /* shared-memory stage/path tables per model (0: global) */
    int max_paths[NUM_MODELS] = {};        /* most scenarios of a tree, per model */
    bool host_inputs = false;            /* staging holds the inputs of the last upload */
    Layout L{};
    char *data = nullptr;
    float *scr = nullptr;
    size_t data_bytes = 0, scr_bytes = 0;
    char *stage = nullptr;
    size_t stage_bytes = 0;
    bool own_stage = false;
    cudaStream_t stream = nullptr;
    cudaStream_t aux[NUM_MODELS] = {};   /* per-model streams of mixed batches */
    cudaEvent_t fork = nullptr, join[NUM_MODELS] = {};
    cudaEvent_t handoff = nullptr;       /* orders a new stream after the old one (bmpc_set_stream) */
    bool any_edge = false;               /* some problem has per-edge dynamics */
    int sm_count = 148;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bmpc_opts gopts{};
    bool have_graph = false;
};

namespace {

void compute_layout(const bmpc_tree_desc *descs, int n, std::vector<ProbRec> &recs, std::vector<int> &nodes,
                    Layout &L) {
    recs.assign(n, ProbRec{});
    nodes.resize(n);
    size_t oi = 0, oin = 0, ow = 0, oo = 0, os = 0;
    int64_t fn = 0, fnx = 0, fnc = 0, fobs = 0;
    for (int k = 0; k < n; ++k) {
        const bmpc_tree_desc &d = descs[k];
        ProbRec &R = recs[k];
        std::memset(&R, 0, sizeof R);
        int max_stage = 0, n_paths = 0, n_bstage = 0;
        {
            std::vector<int> stage;
            validate(d, &stage);
            max_stage = stage.back();
            std::vector<int> nch(d.num_nodes, 0);
            for (int i = 1; i < d.num_nodes; ++i) nch[d.parent[i]]++;
            std::vector<char> bst(max_stage + 1, 0);
            for (int i = 0; i < d.num_nodes; ++i) {
                if (nch[i] == 0) ++n_paths;
                if (nch[i] > 1) bst[stage[i]] = 1;
            }
            for (int s = 0; s <= max_stage; ++s) n_bstage += bst[s];
        }
        R.n = d.num_nodes;
        R.npad = round_up(d.num_nodes, 32);
        R.nx = d.nx;
        R.nu = d.nu;
        R.model = d.model;
        R.n_obs = d.n_obs;
        R.nc = n_con(d);
        R.box_on = d.box_on ? 1 : 0;
        R.lane_on = d.lane_on ? 1 : 0;
        R.n_stage = max_stage + 1;
        R.n_paths = n_paths;
        R.n_bstage = n_bstage;
        R.edge_dyn = d.edge_dynamics;
        {
            Segments sg;
            segments(d.num_nodes, d.parent, sg);
            R.n_waves = (int32_t)sg.wmax.size();
        }
        R.dt = d.dt;
        std::memcpy(R.params, d.params, sizeof R.params);
        R.off_int = (int64_t)oi;
        R.off_in = (int64_t)oin;
        R.off_warm = (int64_t)ow;
        R.off_out = (int64_t)oo;
        R.off_scr = (int64_t)os;
        R.off_node = fn;
        R.off_nx = fnx;
        R.off_nc = fnc;
        R.off_obs = fobs;
        fn += R.n;
        fnx += (int64_t)R.n * R.nx;
        fnc += (int64_t)R.n * R.nc;
        fobs += (int64_t)R.n * R.n_obs * 5;
        oi += (size_t)int_off(R.npad, R.n_stage, R.n_paths, R.n_waves).total;
        oin += (size_t)in_rows(R.nx, R.n_obs, R.edge_dyn).total * R.npad;
        ow += 2 * (size_t)warm_rows(R.nx, R.nc).total * R.npad;   /* primary and fallback slots */
        oo += (size_t)out_rows(R.nx, R.nc).total * R.npad;
        os += (size_t)scr_rows(R.nx).total * R.npad;
        nodes[k] = d.num_nodes;
    }
    L.ints_n = oi;
    L.in_n = oin;
    L.warm_n = ow;
    L.out_n = oo;
    L.scr_n = os;
    L.T_n = fn;
    L.T_nx = fnx;
    L.T_nc = fnc;
    L.T_obs = fobs;
    L.raw_n = (size_t)std::max(fnx + fn + fobs, 2 * fnx + 2 * fn + fnc);
    size_t off = 0;
    L.recs = off;
    off = align_up(off + sizeof(ProbRec) * n);
    L.order = off;
    off = align_up(off + sizeof(int32_t) * n);
    L.queue = off;
    off = align_up(off + sizeof(int32_t) * 4);
    L.ints = off;
    off = align_up(off + sizeof(int32_t) * oi);
    L.in = off;
    off = align_up(off + sizeof(float) * oin);
    L.warm = off;
    off = align_up(off + sizeof(float) * ow);
    L.out = off;
    off = align_up(off + sizeof(float) * oo);
    L.stats = off;
    off = align_up(off + sizeof(Stats) * n);
    /* staging mirrors [recs .. stats] of the data arena; the raw region (flat transfers) is device only */
    L.staging = off;
    L.raw = off;
    off = align_up(off + sizeof(float) * L.raw_n);
    L.data_total = off;
}

KOpts to_kopts(const bmpc_opts &o) {
    KOpts k;
    k.max_iters = o.max_iters;
    k.max_outer = o.max_outer;
    k.n_alpha = o.n_alpha;
    k.ls_chunk = o.ls_chunk;
    k.variant = o.variant;
    k.warm_select = o.warm_select;
    k.cap_rule = o.cap_rule;
    k.compensated = o.compensated;
    k.hessian = o.hessian;
    k.eps_tol = o.eps_tol * o.kkt_margin;   /* the kernel's own FP32 tests, with the margin */
    k.tau = o.tau;
    k.omega0 = o.omega0;
    k.eta0 = o.eta0;
    k.a_omega = o.a_omega;
    k.b_omega = o.b_omega;
    k.a_eta = o.a_eta;
    k.b_eta = o.b_eta;
    k.rho0 = o.rho0;
    k.rho_max = o.rho_max;
    k.mu0 = o.mu0;
    k.beta = o.beta;
    k.ls_rel_eps = o.ls_rel_eps;
    k.select_mu = o.select_mu;
    k.select_rho = o.select_rho;
    return k;
}

int check_opts(const bmpc_opts &o) {
    if (o.max_iters < 0 || o.max_outer < 1 || o.n_alpha < 1 || o.n_alpha > 16) return BMPC_ERR_INVALID;
    if (o.ls_chunk < 0 || o.ls_chunk > 16) return BMPC_ERR_INVALID;
    if (!(o.eps_tol > 0.f) || !(o.tau > 1.f) || !(o.rho0 > 0.f) || !(o.rho_max >= o.rho0)) return BMPC_ERR_INVALID;
    if (!(o.beta > 0.f && o.beta < 0.5f) || !(o.mu0 >= 0.f) || !(o.ls_rel_eps >= 0.f)) return BMPC_ERR_INVALID;
    if (o.block_threads != 0 && (o.block_threads < 32 || o.block_threads > max_block_threads() || o.block_threads % 32))
        return BMPC_ERR_INVALID;
    if (o.blocks_per_sm < 0) return BMPC_ERR_INVALID;
    if (o.variant < 0 || o.variant > 5) return BMPC_ERR_INVALID;
    if (o.warm_select < 0 || o.warm_select > 1 || !(o.select_mu >= 0.f) ||
        !(o.select_rho > 0.f)) return BMPC_ERR_INVALID;
    if (o.queue_order < 0 || o.queue_order > 1) return BMPC_ERR_INVALID;
    if (o.cap_rule < 0 || o.cap_rule > 1) return BMPC_ERR_INVALID;
    if (!(o.kkt_margin > 0.f && o.kkt_margin <= 1.f)) return BMPC_ERR_INVALID;
    if (o.compensated < 0 || o.compensated > 1) return BMPC_ERR_INVALID;
    if (o.hessian < 0 || o.hessian > 1) return BMPC_ERR_INVALID;
    for (int m = 0; m < NUM_MODELS; ++m) {
        const int bt = o.block_threads_model[m];
        if (bt != 0 && (bt < 32 || bt > max_block_threads() || bt % 32)) return BMPC_ERR_INVALID;
    }
    if ((o.variant == 0 || o.variant == 3) && o.block_threads != 0 && o.block_threads % 32) return BMPC_ERR_INVALID;
    return BMPC_OK;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? BMPC_OK : BMPC_ERR_CUDA; }

/* Runs f(k) for k in [0, n) on up to 16 host threads (problems are independent in the host
 * packing and unpacking: each writes its own region of the staging buffer or of the outputs). */
template <typename F>
void for_problems(int n, F &&f) {
    const unsigned hw = std::thread::hardware_concurrency();
    const int T = std::min<int>(std::min<unsigned>(hw ? hw : 1u, 16u), std::max(1, n / 64));
    if (T <= 1) {
        for (int k = 0; k < n; ++k) f(k);
        return;
    }
    std::atomic<int> next{0};
    std::vector<std::thread> pool;
    pool.reserve(T);
    for (int t = 0; t < T; ++t)
        pool.emplace_back([&] {
            for (int k; (k = next.fetch_add(1, std::memory_order_relaxed)) < n;) f(k);
        });
    for (std::thread &t : pool) t.join();
}

template <typename T>
T *at(char *base, size_t off) {
    return reinterpret_cast<T *>(base + off);
}

/* The per-problem scalars of a bmpc_problem (x0, weights, bounds, linear model) into its record. */
void copy_params(ProbRec &R, const bmpc_problem &P) {
    for (int j = 0; j < R.nx; ++j) {
        R.x0[j] = P.x0[j];
        R.Qw[j] = P.Qw[j];
        R.QNw[j] = P.QNw[j];
    }
    for (int j = 0; j < NU; ++j) {
        R.Rw[j] = P.Rw[j];
        R.u_lo[j] = P.u_lo[j];
        R.u_hi[j] = P.u_hi[j];
    }
    R.lane_lo = P.lane_lo;
    R.lane_hi = P.lane_hi;
    if (R.model == 2 && P.Alin && P.Blin) {
        std::memcpy(R.Alin, P.Alin, sizeof(float) * R.nx * R.nx);
        std::memcpy(R.Blin, P.Blin, sizeof(float) * R.nx * NU);
    }
}

FlatArgs flat_args(bmpc_batch *b) {
    FlatArgs f{};
    f.recs = at<const ProbRec>(b->data, b->L.recs);
    f.inbase = at<float>(b->data, b->L.in);
    f.outbase = at<const float>(b->data, b->L.out);
    f.raw = at<float>(b->data, b->L.raw);
    f.T_n = b->L.T_n;
    f.T_nx = b->L.T_nx;
    f.T_nc = b->L.T_nc;
    f.T_obs = b->L.T_obs;
    return f;
}

/* Launch geometry for the problems of one model: threads per problem and persistent blocks. */
void geometry(const bmpc_batch *b, const bmpc_opts &o, int model, int count, int *grid, int *block) {
    int bt = o.block_threads_model[model] ? o.block_threads_model[model] : o.block_threads;
    if (bt == 0) bt = count == 1 ? 128 : 32;
    int per_sm = o.blocks_per_sm;
    if (per_sm == 0) {
        int occ = 1, ld;
        const size_t smem = solve_smem(model, b->tab_ints[model], b->max_paths[model], bt, &ld);
        if (occupancy(model, bt, smem, &occ, to_kopts(o)) != cudaSuccess || occ < 1) occ = 1;
        per_sm = occ;
    }
    *block = bt;
    *grid = std::max(1, std::min(count, b->sm_count * per_sm));
}

int launch(bmpc_batch *b, const bmpc_opts &o) {
    if (o.variant >= 3 && b->any_edge) return BMPC_ERR_INVALID;   /* per-edge dynamics: sweeps 1 and 2 */
    if (o.hessian && (o.variant == 3 || o.variant == 4)) return BMPC_ERR_INVALID;   /* diagonal-cost sweeps */
    KernelArgs a;
    a.recs = at<const ProbRec>(b->data, b->L.recs);
    a.ibase = at<const int32_t>(b->data, b->L.ints);
    a.inbase = at<const float>(b->data, b->L.in);
    a.warmbase = at<const float>(b->data, b->L.warm);
    a.outbase = at<float>(b->data, b->L.out);
    a.scr = b->scr;
    a.stats = at<Stats>(b->data, b->L.stats);
    a.opts = to_kopts(o);
    int32_t *queue = at<int32_t>(b->data, b->L.queue);
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int32_t) * 4, b->stream);
    if (e != cudaSuccess) return BMPC_ERR_CUDA;
    /* one persistent kernel per model; with several models the kernels run concurrently on forked
       streams, so that the blocks of one fill the tail of the other */
    int models = 0;
    for (int m = 0; m < NUM_MODELS; ++m) models += b->model_begin[m + 1] > b->model_begin[m];
    if (models > 1 && cudaEventRecord(b->fork, b->stream) != cudaSuccess) return BMPC_ERR_CUDA;
    bool first = true;
    for (int m = 0; m < NUM_MODELS; ++m) {
        const int cnt = b->model_begin[m + 1] - b->model_begin[m];
        if (cnt == 0) continue;
        cudaStream_t s = b->stream;
        if (models > 1 && !first) {
            s = b->aux[m];
            if (cudaStreamWaitEvent(s, b->fork, 0) != cudaSuccess) return BMPC_ERR_CUDA;
        }
        int32_t *ord = at<int32_t>(b->data, b->L.order) + b->model_begin[m];
        if (o.queue_order == 1 && launch_order(a.recs, a.stats, ord, cnt, s) != cudaSuccess) return BMPC_ERR_CUDA;
        a.order = ord;
        a.n_problems = cnt;
        a.queue = queue + m;
        a.tab_ints = b->tab_ints[m];
        int grid, block;
        geometry(b, o, m, cnt, &grid, &block);
        const size_t smem = solve_smem(m, b->tab_ints[m], b->max_paths[m], block, &a.stg_ld);
        if (launch_solve(a, m, grid, block, smem, s) != cudaSuccess) return BMPC_ERR_CUDA;
        if (s != b->stream &&
            (cudaEventRecord(b->join[m], s) != cudaSuccess || cudaStreamWaitEvent(b->stream, b->join[m], 0) != cudaSuccess))
            return BMPC_ERR_CUDA;
        first = false;
    }
    return BMPC_OK;
}

}  // namespace

extern "C" {

void bmpc_default_opts(bmpc_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->max_iters = 50;
    o->max_outer = 60;
    o->n_alpha = 10;
    o->eps_tol = 1e-5f;
    o->tau = 100.f;
    o->omega0 = 1.f;
    o->eta0 = 0.1f;
    o->a_omega = 1.f;
    o->b_omega = 1.f;
    o->a_eta = 0.1f;
    o->b_eta = 0.9f;
    o->rho0 = 10.f;
    o->rho_max = 1e6f;
    o->mu0 = 1.f;
    o->beta = 1e-4f;
    o->ls_rel_eps = 1e-6f;
    o->ls_chunk = 2;
    o->block_threads = 0;
    o->blocks_per_sm = 0;
    o->variant = 0;
    o->warm_select = 0;
    o->select_mu = 100.f;
    o->select_rho = 1e4f;
    o->queue_order = 1;
    for (int m = 0; m < NUM_MODELS; ++m) o->block_threads_model[m] = 0;
    o->cap_rule = 0;
    o->kkt_margin = 0.8f;
    o->compensated = 1;
    o->hessian = 0;
}

int bmpc_batch_bytes(const bmpc_tree_desc *descs, int32_t n, size_t *data_bytes, size_t *scratch_bytes,
                     size_t *staging_bytes) {
    if (!descs || n < 1) return BMPC_ERR_INVALID;
    for (int k = 0; k < n; ++k)
        if (validate(descs[k], nullptr) != BMPC_OK) return BMPC_ERR_INVALID;
    std::vector<ProbRec> recs;
    std::vector<int> nodes;
    Layout L;
    compute_layout(descs, n, recs, nodes, L);
    if (data_bytes) *data_bytes = L.data_total;
    if (scratch_bytes) *scratch_bytes = std::max<size_t>(kAlign, L.scr_n * sizeof(float));
    if (staging_bytes) *staging_bytes = L.staging;
    return BMPC_OK;
}

int bmpc_create_batch(const bmpc_tree_desc *descs, int32_t n, void *dev_data, size_t data_bytes, void *dev_scratch,
                      size_t scratch_bytes, void *host_staging, size_t staging_bytes, void *stream,
                      bmpc_batch **out) {
    if (!out) return BMPC_ERR_INVALID;
    *out = nullptr;
    size_t need_d, need_s, need_h;
    int st = bmpc_batch_bytes(descs, n, &need_d, &need_s, &need_h);
    if (st != BMPC_OK) return st;
    if (!dev_data || !dev_scratch) return BMPC_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(dev_data) % kAlign) || (reinterpret_cast<uintptr_t>(dev_scratch) % kAlign))
        return BMPC_ERR_INVALID;
    if (data_bytes < need_d || scratch_bytes < need_s) return BMPC_ERR_SPACE;
    if (host_staging && staging_bytes < need_h) return BMPC_ERR_SPACE;
    bmpc_batch *b = new (std::nothrow) bmpc_batch();
    if (!b) return BMPC_ERR_SPACE;
    b->n = n;
    compute_layout(descs, n, b->recs, b->nodes, b->L);
    for (const ProbRec &r : b->recs) b->any_edge = b->any_edge || r.edge_dyn != 0;
    b->data = static_cast<char *>(dev_data);
    b->scr = static_cast<float *>(dev_scratch);
    b->data_bytes = data_bytes;
    b->scr_bytes = scratch_bytes;
    b->stream = static_cast<cudaStream_t>(stream);
    if (host_staging) {
        b->stage = static_cast<char *>(host_staging);
        b->stage_bytes = staging_bytes;
    } else {
        b->stage = static_cast<char *>(std::malloc(need_h));
        if (!b->stage) {
            delete b;
            return BMPC_ERR_SPACE;
        }
        b->stage_bytes = need_h;
        b->own_stage = true;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    /* visiting order: grouped by model (one kernel each), largest trees first within a model
       (longest-processing-time-first on the work queue) */
    b->order.resize(n);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) {
        if (b->recs[a].model != b->recs[c].model) return b->recs[a].model < b->recs[c].model;
        return b->nodes[a] > b->nodes[c];
    });
    for (int m = 0; m <= NUM_MODELS; ++m) b->model_begin[m] = 0;
    for (int k = 0; k < n; ++k) b->model_begin[b->recs[k].model + 1]++;
    for (int m = 0; m < NUM_MODELS; ++m) b->model_begin[m + 1] += b->model_begin[m];
    /* tables of up to 32 KB per problem go to shared memory (below the 48 KB needing no opt-in) */
    for (int k = 0; k < n; ++k) {
        const ProbRec &r = b->recs[k];
        const int64_t t = table_ints(r.npad, r.n_stage, r.n_paths);
        b->tab_ints[r.model] = (int)std::max<int64_t>(b->tab_ints[r.model], t);
        b->max_paths[r.model] = std::max(b->max_paths[r.model], r.n_paths);
    }
    for (int m = 0; m < NUM_MODELS; ++m) {
        if (b->tab_ints[m] > 8192) b->tab_ints[m] = 0;
        if (b->model_begin[m + 1] == b->model_begin[m]) continue;
        size_t most = 0;   /* the largest launch over every allowed block size */
        for (int bt = 32; bt <= max_block_threads(); bt += 32) {
            int ld;
            most = std::max(most, solve_smem(m, b->tab_ints[m], b->max_paths[m], bt, &ld));
        }
        if (prepare_solve(m, most) != cudaSuccess) {
            bmpc_destroy_batch(b);
            return BMPC_ERR_CUDA;
        }
    }
    if (cudaEventCreateWithFlags(&b->handoff, cudaEventDisableTiming) != cudaSuccess) {
        bmpc_destroy_batch(b);
        return BMPC_ERR_CUDA;
    }
    int models = 0;
    for (int m = 0; m < NUM_MODELS; ++m) models += b->model_begin[m + 1] > b->model_begin[m];
    if (models > 1) {   /* streams and events of the concurrent per-model launches */
        bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
        for (int m = 0; m < NUM_MODELS && ok; ++m)
            ok = cudaStreamCreateWithFlags(&b->aux[m], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->join[m], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            bmpc_destroy_batch(b);
            return BMPC_ERR_CUDA;
        }
    }
    for (int k = 0; k < n; ++k) b->parents.insert(b->parents.end(), descs[k].parent, descs[k].parent + descs[k].num_nodes);
    /* int tables of every tree, packed into the staging buffer and uploaded once */
    int32_t *ib = at<int32_t>(b->stage, b->L.ints);
    std::memset(ib, 0, sizeof(int32_t) * b->L.ints_n);
    for (int k = 0; k < n; ++k) {
        const bmpc_tree_desc &d = descs[k];
        const ProbRec &R = b->recs[k];
        int32_t *t = ib + R.off_int;
        const int nn = R.n, np = R.npad, ns = R.n_stage, S = R.n_paths;
        const IntOff io = int_off(np, ns, S, R.n_waves);
        {
            Segments sg;
            segments(nn, d.parent, sg);
            std::copy(sg.fnode.begin(), sg.fnode.end(), t + io.fnode);
            std::copy(sg.fend.begin(), sg.fend.end(), t + io.fend);
            std::copy(sg.wstart.begin(), sg.wstart.end(), t + io.wave);
            std::copy(sg.wmax.begin(), sg.wmax.end(), t + io.wave + R.n_waves + 1);
        }
        int32_t *parent = t + io.parent, *nch = t + io.nchild, *fch = t + io.fchild, *stg = t + io.stage;
        int32_t *leaf = t + io.leaf, *owner = t + io.owner, *ss = t + io.sstart, *bst = t + io.bstage;
        int32_t *ptab = t + io.ptab, *pdepth = t + io.pdepth, *ptop = t + io.ptop;
        for (int i = 0; i < nn; ++i) {
            parent[i] = d.parent[i];
            nch[i] = 0;
            fch[i] = 0;
        }
        stg[0] = 0;
        for (int i = 1; i < nn; ++i) {
            const int p = d.parent[i];
            if (nch[p] == 0) fch[p] = i;
            nch[p]++;
            stg[i] = stg[p] + 1;
        }
        for (int i = nn - 1; i >= 0; --i) leaf[i] = nch[i] ? leaf[fch[i]] : i;
        for (int s = 0; s <= ns; ++s) ss[s] = 0;
        for (int i = 0; i < nn; ++i) ss[stg[i] + 1]++;
        for (int s = 0; s < ns; ++s) ss[s + 1] += ss[s];
        /* paths: one per leaf in node order; a node belongs to the path of its first leaf */
        std::vector<int> rank(nn, -1);
        int np_ = 0;
        for (int i = 0; i < nn; ++i)
            if (nch[i] == 0) rank[i] = np_++;
        for (int i = 0; i < nn; ++i) owner[i] = rank[leaf[i]];
        for (int i = 0; i < nn; ++i) {
            if (nch[i] != 0) continue;
            const int s = rank[i];
            pdepth[s] = stg[i];
            for (int k = 0; k < ns; ++k) ptab[(size_t)s * ns + k] = -1;
            int top = 0;
            for (int j = i; j >= 0; j = parent[j]) {
                ptab[(size_t)s * ns + stg[j]] = j;
                if (owner[j] == s) top = stg[j];
                if (j == 0) break;
            }
            ptop[s] = top;
        }
        int nb = 0;
        for (int s = ns - 1; s >= 0; --s) {
            bool branch = false;
            for (int i = ss[s]; i < ss[s + 1]; ++i) branch |= nch[i] > 1;
            if (branch) bst[nb++] = s;
        }
    }
    std::memcpy(b->stage + b->L.order, b->order.data(), sizeof(int32_t) * n);
    cudaError_t e = cudaMemcpyAsync(b->data + b->L.order, b->stage + b->L.order, sizeof(int32_t) * n,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->data + b->L.ints, b->stage + b->L.ints, sizeof(int32_t) * b->L.ints_n,
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->data + b->L.stats, 0, sizeof(Stats) * n, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        bmpc_destroy_batch(b);
        return BMPC_ERR_CUDA;
    }
    *out = b;
    return BMPC_OK;
}

int bmpc_set_problems(bmpc_batch *b, const bmpc_problem *probs) {
    if (!b || !probs) return BMPC_ERR_INVALID;
    const int n = b->n;
    /* validation first (nothing is changed when a problem is invalid) */
    for (int k = 0; k < n; ++k) {
        const bmpc_problem &P = probs[k];
        const ProbRec &R = b->recs[k];
        if (!P.x0 || !P.xref || (R.n_obs > 0 && !P.obs)) return BMPC_ERR_INVALID;
        if (R.model == 2 && !R.edge_dyn && (!P.Alin || !P.Blin)) return BMPC_ERR_INVALID;
        if (R.edge_dyn && (!P.Aedge || !P.Bedge)) return BMPC_ERR_INVALID;
        const bool warm = P.warm_x || P.warm_u || P.warm_lam || P.warm_y;
        if (warm && (!P.warm_x || !P.warm_u || !P.warm_lam || (R.nc > 0 && !P.warm_y))) return BMPC_ERR_INVALID;
        for (int j = 0; j < R.nx; ++j)
            if (!std::isfinite(P.x0[j])) return BMPC_ERR_INVALID;
        for (int j = 0; j < NU; ++j)
            if (!(P.Rw[j] > 0.f)) return BMPC_ERR_INVALID;
    }
    std::atomic<bool> any_warm{false};
    float *fin = at<float>(b->stage, b->L.in);
    float *fw = at<float>(b->stage, b->L.warm);
    for_problems(n, [&](int k) {
        const bmpc_problem &P = probs[k];
        ProbRec &R = b->recs[k];
        const int nn = R.n, np = R.npad, nx = R.nx, nc = R.nc;
        const bool warm = P.warm_x || P.warm_u || P.warm_lam || P.warm_y;
        copy_params(R, P);
        R.has_warm = warm ? 1 : 0;
        if (warm) any_warm.store(true, std::memory_order_relaxed);
        const InRows ir = in_rows(nx, R.n_obs, R.edge_dyn);
        float *base = fin + R.off_in;
        std::memset(base, 0, sizeof(float) * (size_t)ir.total * np);
        if (R.edge_dyn)   /* per-edge matrices: entry (a, c) of the edge into node i at row a*nx+c, column i */
            for (int i = 1; i < nn; ++i) {
                for (int e = 0; e < nx * nx; ++e) base[(size_t)(ir.edge + e) * np + i] = P.Aedge[(size_t)i * nx * nx + e];
                for (int e = 0; e < nx * NU; ++e)
                    base[(size_t)(ir.edge + nx * nx + e) * np + i] = P.Bedge[(size_t)i * nx * NU + e];
            }
        for (int i = 0; i < nn; ++i) {
            for (int j = 0; j < nx; ++j) base[(size_t)(ir.xref + j) * np + i] = P.xref[(size_t)i * nx + j];
            base[(size_t)ir.weight * np + i] = P.weight ? P.weight[i] : 1.f;
            for (int o = 0; o < R.n_obs; ++o) {
                const float *ob = P.obs + ((size_t)i * R.n_obs + o) * 5;   /* cx, cy, heading, a, b */
                float *row = base + (size_t)(ir.obs + OBS_ROWS * o) * np + i;
                row[0] = ob[0];                  /* rows 2..5 are converted on the device */
                row[(size_t)np] = ob[1];
                row[2 * (size_t)np] = ob[2];
                row[4 * (size_t)np] = ob[3];
                row[5 * (size_t)np] = ob[4];
            }
        }
        if (warm) {
            const WarmRows wr = warm_rows(nx, nc);
            float *wb = fw + R.off_warm;
            std::memset(wb, 0, sizeof(float) * (size_t)wr.total * np);
            for (int i = 0; i < nn; ++i) {
                for (int j = 0; j < nx; ++j) {
                    wb[(size_t)(wr.wx + j) * np + i] = P.warm_x[(size_t)i * nx + j];
                    wb[(size_t)(wr.wl + j) * np + i] = P.warm_lam[(size_t)i * nx + j];
                }
                for (int j = 0; j < NU; ++j) wb[(size_t)(wr.wu + j) * np + i] = P.warm_u[(size_t)i * NU + j];
                for (int c = 0; c < nc; ++c) wb[(size_t)(wr.wy + c) * np + i] = P.warm_y[(size_t)i * nc + c];
            }
        }
    });
    std::memcpy(b->stage + b->L.recs, b->recs.data(), sizeof(ProbRec) * n);
    cudaError_t e = cudaMemcpyAsync(b->data + b->L.recs, b->stage + b->L.recs, sizeof(ProbRec) * n,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->data + b->L.in, b->stage + b->L.in, sizeof(float) * b->L.in_n, cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && b->L.T_obs > 0) e = launch_flat(2, flat_args(b), n, b->stream);
    b->host_inputs = e == cudaSuccess;
    if (e == cudaSuccess && any_warm.load())
        e = cudaMemcpyAsync(b->data + b->L.warm, b->stage + b->L.warm, sizeof(float) * b->L.warm_n,
                            cudaMemcpyHostToDevice, b->stream);
    return cuda_status(e);
}

int bmpc_set_problems_flat(bmpc_batch *b, const bmpc_problem *probs, const float *xref, const float *weight,
                           const float *obs) {
    if (!b || !probs || !xref || (b->L.T_obs > 0 && !obs)) return BMPC_ERR_INVALID;
    const int n = b->n;
    for (int k = 0; k < n; ++k) {
        const bmpc_problem &P = probs[k];
        const ProbRec &R = b->recs[k];
        if (!P.x0 || (R.model == 2 && (!P.Alin || !P.Blin))) return BMPC_ERR_INVALID;
        if (R.edge_dyn) return BMPC_ERR_INVALID;   /* per-edge matrices travel with bmpc_set_problems only */
        for (int j = 0; j < R.nx; ++j)
            if (!std::isfinite(P.x0[j])) return BMPC_ERR_INVALID;
        for (int j = 0; j < NU; ++j)
            if (!(P.Rw[j] > 0.f)) return BMPC_ERR_INVALID;
    }
    for (int k = 0; k < n; ++k) {
        copy_params(b->recs[k], probs[k]);
        b->recs[k].has_warm = 0;
    }
    std::memcpy(b->stage + b->L.recs, b->recs.data(), sizeof(ProbRec) * n);
    FlatArgs f = flat_args(b);
    f.has_weight = weight != nullptr;
    float *raw = at<float>(b->data, b->L.raw);
    cudaError_t e = cudaMemcpyAsync(b->data + b->L.recs, b->stage + b->L.recs, sizeof(ProbRec) * n,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(raw, xref, sizeof(float) * b->L.T_nx, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess && weight)
        e = cudaMemcpyAsync(raw + b->L.T_nx, weight, sizeof(float) * b->L.T_n, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess && b->L.T_obs > 0)
        e = cudaMemcpyAsync(raw + b->L.T_nx + b->L.T_n, obs, sizeof(float) * b->L.T_obs, cudaMemcpyDefault,
                            b->stream);
    if (e == cudaSuccess) e = launch_flat(0, f, n, b->stream);
    b->host_inputs = false;
    return cuda_status(e);
}

int bmpc_solve_batch(bmpc_batch *b, const bmpc_opts *opts) {
    if (!b) return BMPC_ERR_INVALID;
    bmpc_opts o;
    if (opts) o = *opts;
    else bmpc_default_opts(&o);
    int st = check_opts(o);
    if (st != BMPC_OK) return st;
    return launch(b, o);
}

int bmpc_solve_batch_graph(bmpc_batch *b, const bmpc_opts *opts) {
    if (!b) return BMPC_ERR_INVALID;
    bmpc_opts o;
    if (opts) o = *opts;
    else bmpc_default_opts(&o);
    int st = check_opts(o);
    if (st != BMPC_OK) return st;
    if (!b->have_graph || std::memcmp(&o, &b->gopts, sizeof o) != 0) {
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->gexec = nullptr;
        b->graph = nullptr;
        b->have_graph = false;
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return BMPC_ERR_CUDA;
        cudaStream_t saved = b->stream;
        b->stream = cap;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        int ls = BMPC_OK;
        if (e == cudaSuccess) ls = launch(b, o);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        b->stream = saved;
        cudaStreamDestroy(cap);
        if (e != cudaSuccess || e2 != cudaSuccess || ls != BMPC_OK || !g) {
            if (g) cudaGraphDestroy(g);
            return BMPC_ERR_CUDA;
        }
        if (cudaGraphInstantiate(&b->gexec, g, 0) != cudaSuccess) {
            cudaGraphDestroy(g);
            return BMPC_ERR_CUDA;
        }
        b->graph = g;
        b->gopts = o;
        b->have_graph = true;
    }
    return cuda_status(cudaGraphLaunch(b->gexec, b->stream));
}

namespace {
int upload_recs(bmpc_batch *b) {
    std::memcpy(b->stage + b->L.recs, b->recs.data(), sizeof(ProbRec) * b->n);
    return cuda_status(cudaMemcpyAsync(b->data + b->L.recs, b->stage + b->L.recs, sizeof(ProbRec) * b->n,
                                       cudaMemcpyHostToDevice, b->stream));
}
WarmArgs warm_args(bmpc_batch *b, int slot) {
    WarmArgs w{};
    w.recs = at<const ProbRec>(b->data, b->L.recs);
    w.ibase = at<const int32_t>(b->data, b->L.ints);
    w.inbase = at<const float>(b->data, b->L.in);
    w.warmbase = at<float>(b->data, b->L.warm);
    w.order = at<const int32_t>(b->data, b->L.order);
    w.n_problems = b->n;
    w.slot = slot;
    return w;
}
}  // namespace

int bmpc_set_warm_start_device(bmpc_batch *b, const float *dev_start, int64_t stride, int32_t slot) {
    if (!b || !dev_start || slot < 0 || slot > 1) return BMPC_ERR_INVALID;
    for (int k = 0; k < b->n; ++k) {
        const ProbRec &R = b->recs[k];
        if ((int64_t)R.n * (2 * R.nx + NU + R.nc) > stride) return BMPC_ERR_INVALID;
    }
    WarmArgs w = warm_args(b, slot);
    w.src = dev_start;
    w.stride = stride;
    for (ProbRec &R : b->recs) R.has_warm |= 1 << slot;
    int st = upload_recs(b);
    if (st != BMPC_OK) return st;
    return cuda_status(launch_scatter_warm(w, b->stream));
}

int bmpc_shift_warm_start(bmpc_batch *next, const bmpc_batch *prev, int32_t slot) {
    if (!next || !prev || slot < 0 || slot > 1 || next->n != prev->n) return BMPC_ERR_INVALID;
    if (next->parents != prev->parents) return BMPC_ERR_INVALID;
    for (int k = 0; k < next->n; ++k)
        if (next->recs[k].edge_dyn) return BMPC_ERR_INVALID;   /* the shift rolls out per-node dynamics */
    for (int k = 0; k < next->n; ++k)
        if (next->recs[k].model != prev->recs[k].model || next->recs[k].nc != prev->recs[k].nc ||
            next->recs[k].npad != prev->recs[k].npad)
            return BMPC_ERR_INVALID;
    WarmArgs w = warm_args(next, slot);
    w.prev_recs = at<const ProbRec>(prev->data, prev->L.recs);
    w.prev_ibase = at<const int32_t>(prev->data, prev->L.ints);
    w.prev_inbase = at<const float>(prev->data, prev->L.in);
    w.prev_outbase = at<const float>(prev->data, prev->L.out);
    for (ProbRec &R : next->recs) R.has_warm |= 1 << slot;
    int st = upload_recs(next);
    if (st != BMPC_OK) return st;
    for (int m = 0; m < NUM_MODELS; ++m) {
        const int cnt = next->model_begin[m + 1] - next->model_begin[m];
        if (!cnt) continue;
        WarmArgs wm = w;
        wm.order = at<const int32_t>(next->data, next->L.order) + next->model_begin[m];
        wm.n_problems = cnt;
        if (launch_shift_warm(wm, m, next->stream) != cudaSuccess) return BMPC_ERR_CUDA;
    }
    return BMPC_OK;
}

namespace {
GlueArgs glue_args(const bmpc_batch *b) {
    GlueArgs g{};
    g.recs = reinterpret_cast<const ProbRec *>(b->data + b->L.recs);
    g.ibase = reinterpret_cast<const int32_t *>(b->data + b->L.ints);
    g.inbase = reinterpret_cast<const float *>(b->data + b->L.in);
    g.outbase = reinterpret_cast<const float *>(b->data + b->L.out);
    return g;
}
}  // namespace

int bmpc_mlp_features(const bmpc_batch *b, float *feat, int32_t dim, int32_t n_scen, int32_t n_obs_max) {
    if (!b || !feat || n_scen < 0 || n_obs_max < 0) return BMPC_ERR_INVALID;
    for (const ProbRec &R : b->recs)
        if (dim < R.nx - 1 + 5 * n_scen * n_obs_max) return BMPC_ERR_INVALID;
    GlueArgs g = glue_args(b);
    g.out = feat;
    g.stride = dim;
    g.n_scen = n_scen;
    g.n_obs_max = n_obs_max;
    return cuda_status(launch_glue(0, g, b->n, b->stream, 0));
}

int bmpc_mlp_targets(const bmpc_batch *b, float *tgt, int64_t stride, int32_t y_sqrt) {
    if (!b || !tgt || y_sqrt < 0 || y_sqrt > 1) return BMPC_ERR_INVALID;
    for (const ProbRec &R : b->recs)
        if ((int64_t)R.n * (2 * R.nx + NU + R.nc) > stride) return BMPC_ERR_INVALID;
    GlueArgs g = glue_args(b);
    g.out = tgt;
    g.stride = stride;
    g.y_sqrt = y_sqrt;
    return cuda_status(launch_glue(1, g, b->n, b->stream, 0));
}

int bmpc_mlp_start(const bmpc_batch *b, const float *pred, int64_t ld_pred, const float *mean, const float *std,
                   float *start, int64_t stride, int32_t y_sqrt) {
    if (!b || !pred || !mean || !std || !start || y_sqrt < 0 || y_sqrt > 1) return BMPC_ERR_INVALID;
    for (const ProbRec &R : b->recs)
        if (R.edge_dyn) return BMPC_ERR_INVALID;   /* the rollout of the start uses per-node dynamics */
    for (const ProbRec &R : b->recs) {
        const int64_t used = (int64_t)R.n * (2 * R.nx + NU + R.nc);
        if (used > stride || used > ld_pred) return BMPC_ERR_INVALID;
    }
    GlueArgs g = glue_args(b);
    g.out = start;
    g.stride = stride;
    g.pred = pred;
    g.ld_pred = ld_pred;
    g.mean = mean;
    g.std = std;
    g.y_sqrt = y_sqrt;
    for (int m = 0; m < NUM_MODELS; ++m) {
        const int cnt = b->model_begin[m + 1] - b->model_begin[m];
        g.order_base = reinterpret_cast<const int32_t *>(b->data + b->L.order) + b->model_begin[m];
        if (launch_glue(2, g, cnt, b->stream, m) != cudaSuccess) return BMPC_ERR_CUDA;
    }
    return BMPC_OK;
}

int bmpc_autotune(bmpc_batch *b, const bmpc_opts *base, bmpc_opts *best, float *best_us_per_solve) {
    if (!b || !best) return BMPC_ERR_INVALID;
    bmpc_opts o;
    if (base) o = *base;
    else bmpc_default_opts(&o);
    int st = check_opts(o);
    if (st != BMPC_OK) return st;
    static const int kThreads[] = {32, 64, 128, 256, 512};
    static const int kVariant[] = {1, 2, 3, 4, 5};
    static const int kChunk[] = {1, 2, 4};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return BMPC_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return BMPC_ERR_CUDA;
    }
    std::vector<Stats> stats(b->n);
    double best_rate = -1.0;
    bmpc_opts best_o = o;
    float best_ms = 0.f;
    int rc = BMPC_OK;
    /* converged solves per ms of configuration c (one warm-up launch, one timed); -1 on a CUDA error */
    auto trial = [&](const bmpc_opts &c, float *ms_out) -> double {
        if (launch(b, c) != BMPC_OK) return -1.0;
        if (cudaEventRecord(e0, b->stream) != cudaSuccess || launch(b, c) != BMPC_OK ||
            cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
            return -1.0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (cudaMemcpy(stats.data(), b->data + b->L.stats, sizeof(Stats) * b->n, cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return -1.0;
        int conv = 0;
        for (const Stats &s : stats) conv += s.status == BMPC_OK;
        *ms_out = ms;
        return ms > 0.f ? conv / (double)ms : 0.0;
    };
    for (int bt : kThreads)
        for (int v : kVariant)
            for (int ch : kChunk) {
                if (v >= 3 && b->any_edge) continue;   /* per-edge dynamics: sweeps 1 and 2 */
                if (o.hessian && (v == 3 || v == 4)) continue;
                if (v == 4 && b->n > 1) continue;   /* scan sweeps: single latency-critical solves */
                bmpc_opts c = o;
                c.block_threads = bt;
                for (int m = 0; m < NUM_MODELS; ++m) c.block_threads_model[m] = 0;
                c.variant = v;
                c.ls_chunk = ch;
                c.blocks_per_sm = 0;
                float ms = 0.f;
                const double rate = trial(c, &ms);
                if (rate < 0.0) { rc = BMPC_ERR_CUDA; goto out; }
                if (rate > best_rate) {
                    best_rate = rate;
                    best_o = c;
                    best_ms = ms;
                }
            }
    /* mixed batches: then the threads per problem of each model's launch, one model at a time */
    {
        int models = 0;
        for (int m = 0; m < NUM_MODELS; ++m) models += b->model_begin[m + 1] > b->model_begin[m];
        for (int m = 0; m < NUM_MODELS && models > 1; ++m) {
            if (b->model_begin[m + 1] == b->model_begin[m]) continue;
            const bmpc_opts base_o = best_o;
            for (int bt : kThreads) {
                if (bt == base_o.block_threads) continue;
                bmpc_opts c = base_o;
                c.block_threads_model[m] = bt;
                float ms = 0.f;
                const double rate = trial(c, &ms);
                if (rate < 0.0) { rc = BMPC_ERR_CUDA; goto out; }
                if (rate > best_rate) {
                    best_rate = rate;
                    best_o = c;
                    best_ms = ms;
                }
            }
        }
    }
out:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != BMPC_OK) return rc;
    *best = best_o;
    if (best_us_per_solve) *best_us_per_solve = best_ms * 1e3f / (float)b->n;
    return BMPC_OK;
}

/* Public statistics from the device records copied into the staging area. */
static void stats_from_stage(const bmpc_batch *b, bmpc_stats *stats) {
    const Stats *s = at<const Stats>(b->stage, b->L.stats);
    for (int k = 0; k < b->n; ++k) {
        stats[k].status = s[k].status;
        stats[k].inner_iters = s[k].inner_iters;
        stats[k].outer_iters = s[k].outer_iters;
        stats[k].ls_fail_total = s[k].ls_fail_total;
        stats[k].ls_evals = s[k].ls_evals;
        stats[k].start_used = s[k].start_used;
        stats[k].r_kkt = s[k].r_kkt;
        stats[k].c = s[k].c;
        stats[k].rho = s[k].rho;
        stats[k].mu = s[k].mu;
        stats[k].cycles_linearise = s[k].cyc_lin;
        stats[k].cycles_backward = s[k].cyc_bwd;
        stats[k].cycles_forward = s[k].cyc_fwd;
        stats[k].cycles_linesearch = s[k].cyc_ls;
        stats[k].cycles_total = s[k].cyc_total;
    }
}

int bmpc_get_solutions(bmpc_batch *b, float *x, float *u, float *lam, float *y, bmpc_stats *stats) {
    if (!b) return BMPC_ERR_INVALID;
    cudaError_t e = cudaSuccess;
    if (x && !b->host_inputs) {   /* absolute states need the references of the last upload */
        e = cudaMemcpyAsync(b->stage + b->L.in, b->data + b->L.in, sizeof(float) * b->L.in_n,
                            cudaMemcpyDeviceToHost, b->stream);
        b->host_inputs = e == cudaSuccess;
    }
    if (e == cudaSuccess && (x || u || lam || y))
        e = cudaMemcpyAsync(b->stage + b->L.out, b->data + b->L.out, sizeof(float) * b->L.out_n,
                            cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->stage + b->L.stats, b->data + b->L.stats, sizeof(Stats) * b->n,
                            cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return BMPC_ERR_CUDA;
    const float *fo = at<const float>(b->stage, b->L.out);
    const float *fi = at<const float>(b->stage, b->L.in);
    std::vector<size_t> offx(b->n + 1, 0), offu(b->n + 1, 0), offy(b->n + 1, 0);   /* node-major offsets */
    for (int k = 0; k < b->n; ++k) {
        const ProbRec &R = b->recs[k];
        offx[k + 1] = offx[k] + (size_t)R.n * R.nx;
        offu[k + 1] = offu[k] + (size_t)R.n * NU;
        offy[k + 1] = offy[k] + (size_t)R.n * R.nc;
    }
    for_problems((x || u || lam || y) ? b->n : 0, [&](int k) {
        const ProbRec &R = b->recs[k];
        const size_t ox = offx[k], ol = offx[k], ou = offu[k], oy = offy[k];
        const OutRows orw = out_rows(R.nx, R.nc);
        const InRows ir = in_rows(R.nx, R.n_obs);
        const float *base = fo + R.off_out;
        const float *xref = fi + R.off_in + (size_t)ir.xref * R.npad;
        const int nn = R.n, np = R.npad;
        for (int i = 0; i < nn; ++i) {
            for (int j = 0; j < R.nx; ++j) {
                /* the device keeps the deviation from the reference; absolute state on output */
                if (x) x[ox + (size_t)i * R.nx + j] = xref[(size_t)j * np + i] + base[(size_t)(orw.x + j) * np + i];
                if (lam) lam[ol + (size_t)i * R.nx + j] = base[(size_t)(orw.lam + j) * np + i];
            }
            for (int j = 0; j < NU; ++j)
                if (u) u[ou + (size_t)i * NU + j] = base[(size_t)(orw.u + j) * np + i];
            for (int c = 0; c < R.nc; ++c)
                if (y) y[oy + (size_t)i * R.nc + c] = base[(size_t)(orw.y + c) * np + i];
        }
    });
    if (stats) stats_from_stage(b, stats);
    return BMPC_OK;
}

int bmpc_problem_device_outputs(const bmpc_batch *b, int32_t i, float **x, float **u, float **lam, float **y,
                                int32_t *npad) {
    if (!b || i < 0 || i >= b->n) return BMPC_ERR_INVALID;
    const ProbRec &R = b->recs[i];
    const OutRows orw = out_rows(R.nx, R.nc);
    float *base = reinterpret_cast<float *>(b->data + b->L.out) + R.off_out;
    if (x) *x = base + (size_t)orw.x * R.npad;
    if (u) *u = base + (size_t)orw.u * R.npad;
    if (lam) *lam = base + (size_t)orw.lam * R.npad;
    if (y) *y = base + (size_t)orw.y * R.npad;
    if (npad) *npad = R.npad;
    return BMPC_OK;
}

int bmpc_get_solutions_flat_async(bmpc_batch *b, float *x, float *u, float *lam, float *y) {
    if (!b) return BMPC_ERR_INVALID;
    const FlatArgs f = flat_args(b);
    const float *raw = f.raw;
    cudaError_t e = cudaSuccess;
    if (x || u || lam || y) e = launch_flat(1, f, b->n, b->stream);
    const size_t nx = sizeof(float) * (size_t)b->L.T_nx, nu = sizeof(float) * 2 * (size_t)b->L.T_n;
    if (e == cudaSuccess && x && nx) e = cudaMemcpyAsync(x, raw, nx, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess && u && nu) e = cudaMemcpyAsync(u, raw + b->L.T_nx, nu, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess && lam && nx)
        e = cudaMemcpyAsync(lam, raw + b->L.T_nx + 2 * b->L.T_n, nx, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess && y && b->L.T_nc)
        e = cudaMemcpyAsync(y, raw + 2 * b->L.T_nx + 2 * b->L.T_n, sizeof(float) * (size_t)b->L.T_nc,
                            cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess)   /* the statistics into the pinned staging area, converted by bmpc_wait_solutions */
        e = cudaMemcpyAsync(b->stage + b->L.stats, b->data + b->L.stats, sizeof(Stats) * b->n,
                            cudaMemcpyDeviceToHost, b->stream);
    return cuda_status(e);
}

int bmpc_wait_solutions(bmpc_batch *b, bmpc_stats *stats) {
    if (!b) return BMPC_ERR_INVALID;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return BMPC_ERR_CUDA;
    if (stats) stats_from_stage(b, stats);
    return BMPC_OK;
}

int bmpc_get_solutions_flat(bmpc_batch *b, float *x, float *u, float *lam, float *y, bmpc_stats *stats) {
    const int st = bmpc_get_solutions_flat_async(b, x, u, lam, y);
    return st != BMPC_OK ? st : bmpc_wait_solutions(b, stats);
}

int bmpc_transfer_bytes_flat(const bmpc_batch *b, size_t *h2d, size_t *d2h) {
    if (!b) return BMPC_ERR_INVALID;
    const size_t T_n = (size_t)b->L.T_n, T_nx = (size_t)b->L.T_nx, T_nc = (size_t)b->L.T_nc;
    if (h2d) *h2d = sizeof(ProbRec) * (size_t)b->n + sizeof(float) * (T_nx + T_n + (size_t)b->L.T_obs);
    if (d2h) *d2h = sizeof(float) * (2 * T_nx + 2 * T_n + T_nc) + sizeof(Stats) * (size_t)b->n;
    return BMPC_OK;
}

int bmpc_transfer_bytes(const bmpc_batch *b, size_t *h2d_cold, size_t *h2d_warm, size_t *d2h) {
    if (!b) return BMPC_ERR_INVALID;
    const size_t cold = sizeof(ProbRec) * (size_t)b->n + sizeof(float) * b->L.in_n;
    if (h2d_cold) *h2d_cold = cold;
    if (h2d_warm) *h2d_warm = cold + sizeof(float) * b->L.warm_n;
    if (d2h) *d2h = sizeof(float) * b->L.out_n + sizeof(Stats) * (size_t)b->n;
    return BMPC_OK;
}

int bmpc_get_queue_order(const bmpc_batch *b, int32_t *order) {
    if (!b || !order) return BMPC_ERR_INVALID;
    if (cudaMemcpyAsync(order, b->data + b->L.order, sizeof(int32_t) * b->n, cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return BMPC_ERR_CUDA;
    return BMPC_OK;
}

void bmpc_destroy_batch(bmpc_batch *b) {
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (int m = 0; m < NUM_MODELS; ++m) {
        if (b->aux[m]) cudaStreamDestroy(b->aux[m]);
        if (b->join[m]) cudaEventDestroy(b->join[m]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->handoff) cudaEventDestroy(b->handoff);
    if (b->own_stage) std::free(b->stage);
    delete b;
}

int bmpc_set_stream(bmpc_batch *b, void *stream) {
    if (!b) return BMPC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (s == b->stream) return BMPC_OK;
    /* the new stream waits for everything already issued on the old one */
    if (cudaEventRecord(b->handoff, b->stream) != cudaSuccess || cudaStreamWaitEvent(s, b->handoff, 0) != cudaSuccess)
        return BMPC_ERR_CUDA;
    b->stream = s;
    return BMPC_OK;
}

int bmpc_tree_bytes(const bmpc_tree_desc *desc, size_t *data_bytes, size_t *scratch_bytes, size_t *staging_bytes) {
    return bmpc_batch_bytes(desc, 1, data_bytes, scratch_bytes, staging_bytes);
}

int bmpc_create_tree(const bmpc_tree_desc *desc, void *dev_data, size_t data_bytes, void *dev_scratch,
                     size_t scratch_bytes, void *host_staging, size_t staging_bytes, void *stream, bmpc_tree **out) {
    return bmpc_create_batch(desc, 1, dev_data, data_bytes, dev_scratch, scratch_bytes, host_staging, staging_bytes,
                             stream, out);
}

int bmpc_set_problem(bmpc_tree *t, const bmpc_problem *problem) { return bmpc_set_problems(t, problem); }

int bmpc_solve(bmpc_tree *t, const bmpc_opts *opts, bmpc_stats *stats) {
    int st = bmpc_solve_batch(t, opts);
    if (st != BMPC_OK || !stats) return st;
    st = bmpc_get_solutions(t, nullptr, nullptr, nullptr, nullptr, stats);
    return st != BMPC_OK ? st : stats->status;
}

int bmpc_get_solution(bmpc_tree *t, float *x, float *u, float *lam, float *y) {
    return bmpc_get_solutions(t, x, u, lam, y, nullptr);
}

void bmpc_destroy_tree(bmpc_tree *t) { bmpc_destroy_batch(t); }

const char *bmpc_status_str(int s) {
    switch (s) {
        case BMPC_OK: return "converged";
        case BMPC_MAX_ITER: return "iteration cap reached";
        case BMPC_LS_FAIL: return "line search failed three times in a row";
        case BMPC_ERR_INVALID: return "invalid argument";
        case BMPC_ERR_CUDA: return "CUDA error";
        case BMPC_ERR_NUMERIC: return "numerical failure (H not positive definite or non-finite value)";
        case BMPC_ERR_TIMEOUT: return "device wait timed out";
        case BMPC_ERR_SPACE: return "arena or staging buffer too small";
        default: return "unknown status";
    }
}

const char *bmpc_version(void) { return "bmpc 0.1 sm_103a fp32"; }

int bmpc_selftest_sincos(const float *a, float *s, float *c, int32_t n, void *stream) {
    if (n < 0 || (n > 0 && (!a || !s || !c))) return BMPC_ERR_INVALID;
    return bmpc::launch_sincos(a, s, c, n, static_cast<cudaStream_t>(stream)) == cudaSuccess ? BMPC_OK
                                                                                            : BMPC_ERR_CUDA;
}

int bmpc_selftest_eig_modify(float *S, int32_t n, int32_t count, void *stream) {
    if (!S || (n != 6 && n != 8) || count < 1) return BMPC_ERR_INVALID;
    return bmpc::launch_eig(S, n, count, static_cast<cudaStream_t>(stream)) == cudaSuccess ? BMPC_OK : BMPC_ERR_CUDA;
}

int bmpc_selftest_dyn_hessian(int32_t model, const float *params, float dt, const float *x, const float *u,
                              const float *mu, float *H, int32_t count, void *stream) {
    if (model < 0 || model >= NUM_MODELS || !params || !x || !u || !mu || !H || count < 1 || !(dt > 0.f))
        return BMPC_ERR_INVALID;
    return bmpc::launch_dynhess(model, params, dt, x, u, mu, H, count, static_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? BMPC_OK
               : BMPC_ERR_CUDA;
}

int bmpc_selftest_fma(float *out, int32_t blocks, int32_t iters, void *stream) {
    if (!out || blocks < 1 || iters < 1) return BMPC_ERR_INVALID;
    return bmpc::launch_fma(out, blocks, iters, static_cast<cudaStream_t>(stream)) == cudaSuccess ? BMPC_OK
                                                                                                 : BMPC_ERR_CUDA;
}

}  // extern "C"
