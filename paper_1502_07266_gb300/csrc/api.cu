// C ABI of libhelm: handle lifetime (single-problem and batch handles),
// validation, the setup bookkeeping (block partition, auxiliary windows,
// quasi-1D problem table) and the GMRES driver.  All arithmetic on the solve
// path runs in the kernels of coeff.cu, factor.cu, sweep.cu, stencil.cu,
// gmres.cu and adjoint.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <thread>
#include <utility>
#include <vector>

#include "gmres_kernels.h"
#include "helm_internal.h"

static thread_local cudaError_t g_last_cuda = cudaSuccess;
void helm_set_cuda_error(cudaError_t e) { g_last_cuda = e; }

cudaError_t ensure_dyn_smem(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> raised;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = raised[std::make_pair(fn, dev)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

namespace {

struct TimedLaunch {
    cudaEvent_t a, b;
    int kind;   // 0 sweep, 1 stencil
    int nrhs;
};

std::vector<TimedLaunch>* pend(helm_ctx* h) {
    if (!h->tpending) h->tpending = new std::vector<TimedLaunch>();
    return static_cast<std::vector<TimedLaunch>*>(h->tpending);
}

void resolve_timing(helm_ctx* h) {
    if (!h->tpending) return;
    auto* v = pend(h);
    for (auto& t : *v) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.b) == cudaSuccess && cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            if (t.kind == 0) {
                h->stats.sweep_launches++;
                h->stats.sweep_ms += ms;
                h->stats.rhs_applied += t.nrhs;
            } else {
                h->stats.stencil_launches++;
                h->stats.stencil_ms += ms;
            }
        }
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    v->clear();
}

void stats_add(helm_ctx* h, int kind, int nrhs, float ms) {
    if (kind == 0) {
        h->stats.sweep_launches++;
        h->stats.sweep_ms += ms;
        h->stats.rhs_applied += nrhs;
    } else {
        h->stats.stencil_launches++;
        h->stats.stencil_ms += ms;
    }
}

// One GMRES iteration (index j of a cycle) captured as a CUDA graph, with the
// events that time its apply and matvec when timing is on.
struct GmGraph {
    cudaGraphExec_t exec;
    cudaEvent_t ev[3];
    long long nlaunch;   // kernels one replay launches
};

void drop_graphs(helm_ctx* h) {
    GmGraph* G = static_cast<GmGraph*>(h->gm_graphs);
    if (G) {
        for (int j = 0; j < h->opts.restart; ++j) {
            if (G[j].exec) cudaGraphExecDestroy(G[j].exec);
            for (auto& e : G[j].ev)
                if (e) cudaEventDestroy(e);
        }
        delete[] G;
    }
    h->gm_graphs = nullptr;
}

int fail_cuda(cudaError_t e) {
    helm_set_cuda_error(e);
    return (e == cudaErrorMemoryAllocation) ? HELM_ENOMEM : HELM_ECUDA;
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

// Blocks of a swept axis in axis order with their roles ('L' lower front,
// 'U' upper front, 'C' the centre block that ends the forward passes).  One
// front: the PML slab [0, b), blocks of d layers, the last one the centre.  Two
// fronts: the PML slabs at both ends, q = (N - 2b - 1) / (2d) blocks of d layers
// from each end, the centre block of the 1..2d layers between them.
struct AxisBlock { int m, e; char role; };
std::vector<AxisBlock> axis_blocks(int N, int b, int d, int sched) {
    std::vector<AxisBlock> out;
    if (sched == HELM_TWO_FRONT) {
        const int q = (N - 2 * b - 1) / (2 * d);
        out.push_back({0, b, 'L'});
        for (int i = 0; i < q; ++i) out.push_back({b + i * d, b + (i + 1) * d, 'L'});
        out.push_back({b + q * d, N - b - q * d, 'C'});
        for (int i = q - 1; i >= 0; --i) out.push_back({N - b - (i + 1) * d, N - b - i * d, 'U'});
        out.push_back({N - b, N, 'U'});
        return out;
    }
    out.push_back({0, b, 'L'});
    for (int m = b; m < N; m += d) out.push_back({m, std::min(m + d, N), 'L'});
    out.back().role = 'C';
    return out;
}

// Swept-axis blocks and their auxiliary windows (identical for x2 and x3): a
// side gets b_aux extra layers with a moving PML when the block's role
// eliminates towards it and the block is not at that face; a window clipped by
// a face keeps that side's global profile.
std::vector<AxisWin> make_windows(int N, int b, int d, int b_aux, int sched) {
    std::vector<AxisWin> w;
    for (const AxisBlock& k : axis_blocks(N, b, d, sched)) {
        AxisWin a;
        a.moving = (k.role != 'U' && k.m > 0) ? 1 : 0;
        a.moving_hi = (k.role != 'L' && k.e < N) ? 1 : 0;
        int lo = a.moving ? k.m - b_aux : k.m;
        int hi = a.moving_hi ? k.e + b_aux : k.e;
        if (lo < 0) { lo = 0; a.moving = 0; }
        if (hi > N) { hi = N; a.moving_hi = 0; }
        a.lo = lo;
        a.L = hi - lo;
        a.ia = k.m - lo;
        a.ib = k.e - lo;
        w.push_back(a);
    }
    return w;
}

void free_ctx(helm_ctx* h) {
    if (!h) return;
    for (int p = 0; p < h->nsub; ++p) free_ctx(h->sub[p]);
    if (h->tpending) {
        resolve_timing(h);
        delete pend(h);
        h->tpending = nullptr;
    }
    dense_free(h);
    drop_graphs(h);
    if (h->gm_cap_stream) cudaStreamDestroy((cudaStream_t)h->gm_cap_stream);
    void* ptrs[] = {h->t.s_node, h->t.s_half, h->t.c_dn, h->t.c_up, h->t.w_node, h->t.w_half,
                    h->t.win, h->t.kappa, h->t.kappa64, h->t.c_dn64, h->t.c_up64, h->t.prob,
                    h->factors, h->slab, h->dev_err, h->gm_buf, h->adj_buf};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete[] h->prob_h;
    delete h;
}

}  // namespace

namespace {

// Batch handles: entries of problem p's vectors, the total right-hand sides.
size_t sub_points(const helm_ctx* s) { return (size_t)s->g.N * s->g.N * s->g.N; }
int batch_total(const helm_ctx* h) {
    int t = 0;
    for (int p = 0; p < h->nsub; ++p) t += h->sub_nrhs[p];
    return t;
}

}  // namespace

void helm_time_begin(helm_ctx* h, cudaStream_t st, void** ev0) {
    *ev0 = nullptr;
    if (!h->timing) return;
    cudaEvent_t a;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    cudaEventRecord(a, st);
    *ev0 = (void*)a;
}

void helm_time_end(helm_ctx* h, cudaStream_t st, void* ev0, int kind, int nrhs) {
    if (!h->timing || !ev0) return;
    cudaEvent_t b;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy((cudaEvent_t)ev0); return; }
    cudaEventRecord(b, st);
    pend(h)->push_back(TimedLaunch{(cudaEvent_t)ev0, b, kind, nrhs});
    if (pend(h)->size() > 4096) resolve_timing(h);
}

extern "C" {

int helm_enable_timing(helm_handle h, int on) {
    if (h && h->nsub) {
        for (int p = 0; p < h->nsub; ++p) helm_enable_timing(h->sub[p], on);
        return HELM_OK;
    }
    if (!h) return HELM_EINVAL;
    h->timing = on ? 1 : 0;
    return HELM_OK;
}

int helm_get_stats(helm_handle h, helm_stats* out) {
    if (!h || !out) return HELM_EINVAL;
    if (h->nsub) {
        helm_stats t;
        memset(&t, 0, sizeof(t));
        for (int p = 0; p < h->nsub; ++p) {
            helm_stats q;
            helm_get_stats(h->sub[p], &q);
            t.sweep_launches += q.sweep_launches;
            t.sweep_ms += q.sweep_ms;
            t.stencil_launches += q.stencil_launches;
            t.stencil_ms += q.stencil_ms;
            t.rhs_applied += q.rhs_applied;
        }
        *out = t;
        return HELM_OK;
    }
    resolve_timing(h);
    *out = h->stats;
    return HELM_OK;
}

void helm_reset_stats(helm_handle h) {
    if (!h) return;
    for (int p = 0; p < h->nsub; ++p) helm_reset_stats(h->sub[p]);
    resolve_timing(h);
    memset(&h->stats, 0, sizeof(h->stats));
}

void helm_default_opts(helm_opts* o) {
    if (!o) return;
    o->precision = HELM_FP32;
    o->b_aux = 0;
    o->restart = 30;
    o->maxit = 300;
    o->pml_C = 10.0;
    o->rhs_per_cta = 0;
    o->schedule = HELM_ONE_FRONT;
    o->apply_form = HELM_CHAIN;
    o->debug_unmet_wait = 0;
    o->wait_cycles = 0;
    o->dense_clusters = 0;
    o->reserved_ = 0;
}

const char* helm_strerror(int code) {
    switch (code) {
        case HELM_OK: return "ok";
        case HELM_ENOCONV: return "GMRES did not reach the tolerance within maxit";
        case HELM_EINVAL: return "invalid argument";
        case HELM_ENOMEM: return "device memory allocation failed";
        case HELM_ECUDA: return "CUDA runtime error";
        case HELM_ETIMEOUT: return "a bounded device wait expired";
        case HELM_ENOTSUP: return "unsupported configuration (quasi-1D block larger than 64)";
        default: return "unknown error";
    }
}

int helm_setup(const float* c, double omega, int n, int b, int d, const helm_opts* opts, void* stream,
               helm_handle* out) {
    if (!out) return HELM_EINVAL;
    *out = nullptr;
    if (!c || n < 1 || b < 1 || d < 1 || !(omega > 0.0) || !isfinite(omega)) return HELM_EINVAL;
    helm_opts o;
    helm_default_opts(&o);
    if (opts) {
        o = *opts;
        if (o.restart <= 0) o.restart = 30;
        if (o.maxit <= 0) o.maxit = 300;
        if (!(o.pml_C > 0.0)) o.pml_C = 10.0;
        if (o.b_aux < 0 || o.rhs_per_cta < 0) return HELM_EINVAL;
        if (o.schedule != HELM_ONE_FRONT && o.schedule != HELM_TWO_FRONT) return HELM_EINVAL;
        if (o.schedule == HELM_TWO_FRONT && (o.apply_form != HELM_DENSE || n - 1 < 2 * d)) return HELM_ENOTSUP;
        if (o.precision != HELM_FP32 && o.precision != HELM_FP16 && o.precision != HELM_SPLIT_FP16)
            return HELM_EINVAL;
        if (o.apply_form != HELM_CHAIN && o.apply_form != HELM_DENSE) return HELM_EINVAL;
        if (o.wait_cycles < 0 || o.debug_unmet_wait < 0 || o.dense_clusters < 0) return HELM_EINVAL;
    }
    const bool dense = o.apply_form == HELM_DENSE;
    if (o.restart > 62) return HELM_EINVAL;
    const int N = n + 2 * b;
    const int b_aux = o.b_aux > 0 ? o.b_aux : b;
    std::vector<AxisWin> win = make_windows(N, b, d, b_aux, o.schedule);
    const int B = (int)win.size();
    int cen = B - 1;
    if (o.schedule == HELM_TWO_FRONT) {
        const std::vector<AxisBlock> blk = axis_blocks(N, b, d, o.schedule);
        for (int q = 0; q < B; ++q)
            if (blk[q].role == 'C') cen = q;
    }
    int Wmax = 0;
    for (auto& w : win) Wmax = std::max(Wmax, w.L);

    std::vector<Prob> prob((size_t)B * B);
    long long off = 0;
    int kmax = 0, se = 0;
    for (int M = 0; M < B; ++M) {
        for (int Mp = 0; Mp < B; ++Mp) {
            Prob& P = prob[(size_t)M * B + Mp];
            const AxisWin& wy = win[Mp];
            const AxisWin& wz = win[M];
            P.Ly = wy.L;
            P.Lz = wz.L;
            P.k = P.Ly * P.Lz;
            if (P.k > HELM_KMAX) return HELM_ENOTSUP;
            P.ylo = wy.lo;
            P.a0 = P.Lz * wy.ia;
            P.ni = P.Lz * (wy.ib - wy.ia);
            P.yb0 = wy.lo + wy.ia;
            P.yb1 = wy.lo + wy.ib;
            // sweep-kernel layout: rows zero padded to a multiple of 8 columns (the
            // product tiles read 8-column chunks without bounds tests), then 2 or 4
            // more entries so that the row stride is an odd number of 16-byte
            // granules: the 8 rows a quarter-warp reads hit distinct banks
            P.hp = (P.k + 1) / 2;
            P.ldk = 8 * ((P.k + 7) / 8) + ((o.precision == HELM_FP16 && !dense) ? 4 : 2);
            P.kstride = P.k * P.ldk;
            P.pad_[0] = P.pad_[1] = 0;
            P.off = off;
            off += (long long)N * P.kstride;
            kmax = std::max(kmax, P.k);
            se = std::max(se, P.kstride);
        }
    }

    helm_ctx* h = new helm_ctx();
    memset(h, 0, sizeof(*h));
    h->opts = o;
    h->g.n = n; h->g.b = b; h->g.d = d; h->g.N = N; h->g.B = B; h->g.b_aux = b_aux;
    h->g.cen = cen;
    h->g.sched = o.schedule;
    h->g.h = 1.0 / (n + 1);
    h->g.omega = omega;
    h->g.C = o.pml_C;
    h->g.Wmax = Wmax;
    h->kmax = kmax;
    h->stage_elems = se;
    h->esz = (o.precision == HELM_FP16 && !dense) ? 4 : 8;
    h->factor_bytes = dense ? 0 : (size_t)off * h->esz;
    h->factor_elems = (h->factor_bytes + sizeof(float2) - 1) / sizeof(float2);
    h->dense = dense ? 1 : 0;
    h->prob_h = new Prob[prob.size()];
    memcpy(h->prob_h, prob.data(), sizeof(Prob) * prob.size());
    cudaGetDevice(&h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n3 = (size_t)N * N * N;

    cudaError_t e = cudaSuccess;
#define TRY(x) do { e = (x); if (e != cudaSuccess) { int rc = fail_cuda(e); free_ctx(h); return rc; } } while (0)
    TRY(dalloc(&h->t.s_node, N));
    TRY(dalloc(&h->t.s_half, N + 1));
    TRY(dalloc(&h->t.c_dn, N));
    TRY(dalloc(&h->t.c_up, N));
    TRY(dalloc(&h->t.c_dn64, N));
    TRY(dalloc(&h->t.c_up64, N));
    TRY(dalloc(&h->t.w_node, (size_t)B * Wmax));
    TRY(dalloc(&h->t.w_half, (size_t)B * (Wmax + 1)));
    TRY(dalloc(&h->t.win, B));
    TRY(dalloc(&h->t.kappa, n3));
    TRY(dalloc(&h->t.kappa64, n3));
    TRY(dalloc(&h->t.prob, (size_t)B * B));
    TRY(dalloc(&h->dev_err, 1));
    if (!dense) TRY(dalloc(&h->factors, h->factor_elems));
    TRY(cudaMemsetAsync(h->dev_err, 0, sizeof(int), st));
    TRY(cudaMemcpyAsync(h->t.win, win.data(), sizeof(AxisWin) * B, cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(h->t.prob, prob.data(), sizeof(Prob) * prob.size(), cudaMemcpyHostToDevice, st));
    TRY(launch_coefficients(h, c, st));
    if (!dense) TRY(launch_factor(h, st));
    int herr = 0;
    TRY(cudaMemcpyAsync(&herr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
#undef TRY
    if (herr & 1) { free_ctx(h); return HELM_EINVAL; }
    int rc = HELM_OK;
    if (dense) {
        rc = dense_setup(h, &win, &prob, st);
        if (rc == HELM_OK) {
            herr = 0;
            cudaError_t e2 = cudaMemcpyAsync(&herr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
            if (e2 != cudaSuccess) rc = fail_cuda(e2);
            else if (herr) rc = HELM_ECUDA;
        }
    } else {
        rc = sweep_configure(h);
    }
    if (rc != HELM_OK) { free_ctx(h); return rc; }
    *out = h;
    return HELM_OK;
}

void helm_destroy(helm_handle h) { free_ctx(h); }

namespace {

// First and last window (inclusive) meeting the node range [lo, hi), or -1.
void windows_meeting(const std::vector<AxisWin>& w, int lo, int hi, int* first, int* last) {
    *first = *last = -1;
    for (int M = 0; M < (int)w.size(); ++M) {
        if (w[M].lo < hi && w[M].lo + w[M].L > lo) {
            if (*first < 0) *first = M;
            *last = M;
        }
    }
}

bool box_ok(const int* box, int N) {
    for (int a = 0; a < 3; ++a)
        if (box[2 * a] < 0 || box[2 * a] >= box[2 * a + 1] || box[2 * a + 1] > N) return false;
    return true;
}

}  // namespace

int helm_affected_problems(int n, int b, int d, int b_aux, int schedule, const int* box, int* out) {
    if (!box || !out || n < 1 || b < 1 || d < 1 || b_aux < 0) return HELM_EINVAL;
    if (schedule != HELM_ONE_FRONT && (schedule != HELM_TWO_FRONT || n - 1 < 2 * d)) return HELM_EINVAL;
    const int N = n + 2 * b;
    if (!box_ok(box, N)) return HELM_EINVAL;
    const std::vector<AxisWin> w = make_windows(N, b, d, b_aux > 0 ? b_aux : b, schedule);
    windows_meeting(w, box[4], box[5], &out[0], &out[1]);   // slabs: z windows
    windows_meeting(w, box[2], box[3], &out[2], &out[3]);   // line blocks: y windows
    return HELM_OK;
}

int helm_update_velocity(helm_handle h, const float* c_new, const int* box, int* nprob_out, void* stream) {
    if (!h || !c_new || !box) return HELM_EINVAL;
    if (h->nsub) return HELM_ENOTSUP;
    const int B = h->g.B;
    int r[4];
    int rc = helm_affected_problems(h->g.n, h->g.b, h->g.d, h->g.b_aux, h->g.sched, box, r);
    if (rc != HELM_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(h->dev_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_coefficients(h, c_new, st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(e);
    if (herr & 1) return HELM_EINVAL;                       // c <= 0 or non-finite: kappa is unusable
    int nprob = 0;
    if (r[0] >= 0 && r[2] >= 0) {
        nprob = (r[1] - r[0] + 1) * (r[3] - r[2] + 1);
        if (h->dense) {
            rc = dense_rebuild(h, r[0], r[1], r[2], r[3], st);
            if (rc != HELM_OK) return rc;
        } else {
            for (int M = r[0]; M <= r[1] && e == cudaSuccess; ++M)
                e = launch_factor_range(h, M * B + r[2], r[3] - r[2] + 1, h->factors, 0, h->opts.precision, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return fail_cuda(e);
        }
    }
    if (nprob_out) *nprob_out = nprob;
    return HELM_OK;
}

int helm_setup_batch(int nprob, const helm_problem* probs, const helm_opts* opts, void* stream,
                     helm_handle* out) {
    if (!out) return HELM_EINVAL;
    *out = nullptr;
    if (!probs || nprob < 1 || nprob > HELM_MAX_BATCH) return HELM_EINVAL;
    for (int p = 0; p < nprob; ++p)
        if (probs[p].nrhs < 1) return HELM_EINVAL;
    helm_ctx* h = new helm_ctx();
    memset(h, 0, sizeof(*h));
    if (opts) h->opts = *opts;
    else helm_default_opts(&h->opts);
    cudaGetDevice(&h->device);
    for (int p = 0; p < nprob; ++p) {
        int rc = helm_setup(probs[p].c, probs[p].omega, probs[p].n, probs[p].b, probs[p].d, opts, stream,
                            &h->sub[p]);
        if (rc != HELM_OK) {
            free_ctx(h);
            return rc;
        }
        h->sub_nrhs[p] = probs[p].nrhs;
        h->nsub = p + 1;
    }
    *out = h;
    return HELM_OK;
}

int helm_grid_size(helm_handle h) { return (h && !h->nsub) ? h->g.N : -1; }
int helm_num_blocks(helm_handle h) { return (h && !h->nsub) ? h->g.B : -1; }
int helm_slab_layers(helm_handle h, int M) {
    if (!h || h->nsub || M < 0 || M >= h->g.B) return -1;
    // window lengths follow the block partition
    std::vector<AxisWin> w = make_windows(h->g.N, h->g.b, h->g.d, h->g.b_aux, h->g.sched);
    return w[M].L;
}
size_t helm_factor_bytes(helm_handle h) {
    if (!h) return 0;
    size_t t = h->factor_bytes + h->dG_bytes + h->dscale_elems * sizeof(float);
    for (int p = 0; p < h->nsub; ++p) t += helm_factor_bytes(h->sub[p]);
    return t;
}
long long helm_launch_count(helm_handle h) {
    if (!h) return -1;
    long long t = h->launches;
    for (int p = 0; p < h->nsub; ++p) t += helm_launch_count(h->sub[p]);
    return t;
}

int helm_apply_precond(helm_handle h, const void* r, void* z, int nrhs, void* stream) {
    if (!h || !r || !z || nrhs < 1) return HELM_EINVAL;
    if (r == z) return HELM_EINVAL;
    if (h->nsub) {                                   // one launch over every problem
        if (nrhs != batch_total(h)) return HELM_EINVAL;
        const void* rp[HELM_MAX_BATCH];
        void* zp[HELM_MAX_BATCH];
        size_t off = 0;
        for (int p = 0; p < h->nsub; ++p) {
            rp[p] = (const float2*)r + off;
            zp[p] = (float2*)z + off;
            off += (size_t)h->sub_nrhs[p] * sub_points(h->sub[p]);
        }
        return helm_apply_batch(h->sub, rp, zp, h->sub_nrhs, h->nsub, stream);
    }
    void* ev;
    helm_time_begin(h, (cudaStream_t)stream, &ev);
    cudaError_t e = launch_sweep(h, (const float2*)r, (float2*)z, nrhs, 0, 0, (cudaStream_t)stream);
    helm_time_end(h, (cudaStream_t)stream, ev, 0, nrhs);
    if (e != cudaSuccess) return fail_cuda(e);
    return HELM_OK;
}

int helm_apply_slab(helm_handle h, int M, const void* g, void* v, int nrhs, void* stream) {
    if (h && (h->nsub || h->dense)) return HELM_ENOTSUP;
    if (!h || !g || !v || nrhs < 1 || M < 0 || M >= h->g.B || g == v) return HELM_EINVAL;
    cudaError_t e = launch_sweep(h, (const float2*)g, (float2*)v, nrhs, 1, M, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e);
    return HELM_OK;
}

int helm_matvec(helm_handle h, const void* x, void* y, int nrhs, int fp64, void* stream) {
    if (!h || !x || !y || nrhs < 1 || x == y) return HELM_EINVAL;
    if (h->nsub) {
        if (nrhs != batch_total(h)) return HELM_EINVAL;
        const size_t es = fp64 ? sizeof(double2) : sizeof(float2);
        size_t off = 0;
        for (int p = 0; p < h->nsub; ++p) {
            int rc = helm_matvec(h->sub[p], (const char*)x + off, (char*)y + off, h->sub_nrhs[p], fp64, stream);
            if (rc != HELM_OK) return rc;
            off += (size_t)h->sub_nrhs[p] * sub_points(h->sub[p]) * es;
        }
        return HELM_OK;
    }
    void* ev;
    helm_time_begin(h, (cudaStream_t)stream, &ev);
    cudaError_t e = fp64 ? launch_stencil_c128(h, (const double2*)x, (double2*)y, nrhs, (cudaStream_t)stream)
                         : launch_stencil_c64(h, (const float2*)x, (float2*)y, nrhs, (cudaStream_t)stream);
    helm_time_end(h, (cudaStream_t)stream, ev, 1, nrhs);
    if (e != cudaSuccess) return fail_cuda(e);
    return HELM_OK;
}

int helm_status(helm_handle h, void* stream) {
    if (!h) return HELM_EINVAL;
    if (h->nsub) {
        int rc = HELM_OK;
        for (int p = 0; p < h->nsub; ++p) {
            int q = helm_status(h->sub[p], stream);
            if (q != HELM_OK && rc == HELM_OK) rc = q;
        }
        return rc;
    }
    int herr = 0;
    cudaError_t e = cudaMemcpyAsync(&herr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e);
    if (herr & 2) return HELM_ETIMEOUT;
    return HELM_OK;
}

int helm_solve(helm_handle h, const void* f_, void* u_, int nrhs, double tol, int* iters, double* relres,
               void* stream) {
    if (!h || !f_ || !u_ || nrhs < 1 || !(tol > 0.0) || f_ == u_) return HELM_EINVAL;
    if (h->nsub) {                                   // the problems' solves run concurrently
        if (nrhs != batch_total(h)) return HELM_EINVAL;
        const void* fp[HELM_MAX_BATCH];
        void* up[HELM_MAX_BATCH];
        size_t off = 0;
        for (int p = 0; p < h->nsub; ++p) {
            fp[p] = (const float2*)f_ + off;
            up[p] = (float2*)u_ + off;
            off += (size_t)h->sub_nrhs[p] * sub_points(h->sub[p]);
        }
        return helm_solve_batch(h->sub, fp, up, h->sub_nrhs, h->nsub, tol, iters, relres, stream);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const float2* f = (const float2*)f_;
    const int R = nrhs, m = h->opts.restart, maxit = h->opts.maxit;
    const long long n3 = (long long)h->g.N * h->g.N * h->g.N;
    const long long vs = (long long)R * n3;   // stride between basis vectors

    // ---- work space layout ----
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
    size_t oV = take(sizeof(float2) * (size_t)(m + 1) * vs);
    size_t oZ = take(sizeof(float2) * (size_t)m * vs);
    size_t oW = take(sizeof(float2) * (size_t)vs);
    size_t oU = take(sizeof(double2) * (size_t)vs);
    size_t oR = take(sizeof(double2) * (size_t)vs);
    size_t oH = take(sizeof(double2) * (size_t)R * m * (m + 1));
    size_t oCs = take(sizeof(double2) * (size_t)R * m);
    size_t oSn = take(sizeof(double2) * (size_t)R * m);
    size_t oG = take(sizeof(double2) * (size_t)R * (m + 1));
    size_t oY = take(sizeof(double2) * (size_t)R * m);
    size_t oT = take(sizeof(double2) * (size_t)R * (m + 1));
    size_t oP = take(sizeof(double2) * (size_t)R * 64 * 8);
    size_t oRn = take(sizeof(double) * R);
    size_t oWn = take(sizeof(double) * R);
    size_t oInv = take(sizeof(double) * R);
    size_t oEst = take(sizeof(double) * R);
    size_t oFn = take(sizeof(double) * R);
    size_t oAct = take(sizeof(int) * R);
    size_t oFrz = take(sizeof(int) * R);
    size_t oMl = take(sizeof(int) * R);
    size_t oIt = take(sizeof(int) * R);
    size_t oNa = take(sizeof(int));
    if (off > h->gm_bytes) {
        if (h->gm_buf) cudaFree(h->gm_buf);
        h->gm_buf = nullptr;
        h->gm_bytes = 0;
        cudaError_t e = cudaMalloc(&h->gm_buf, off);
        if (e != cudaSuccess) return fail_cuda(e);
        h->gm_bytes = off;
    }
    char* base = (char*)h->gm_buf;
    float2* V = (float2*)(base + oV);
    float2* Z = (float2*)(base + oZ);
    float2* w = (float2*)(base + oW);
    double2* u64 = (double2*)(base + oU);
    double2* r64 = (double2*)(base + oR);
    double2* H = (double2*)(base + oH);
    double2* cs = (double2*)(base + oCs);
    double2* sn = (double2*)(base + oSn);
    double2* g = (double2*)(base + oG);
    double2* y = (double2*)(base + oY);
    double2* tmp = (double2*)(base + oT);
    double2* part = (double2*)(base + oP);
    double* rn2 = (double*)(base + oRn);
    double* wn2 = (double*)(base + oWn);
    double* inv = (double*)(base + oInv);
    double* est = (double*)(base + oEst);
    double* fn2 = (double*)(base + oFn);
    int* active = (int*)(base + oAct);
    int* frozen = (int*)(base + oFrz);
    int* mlen = (int*)(base + oMl);
    int* its_d = (int*)(base + oIt);
    int* nact_d = (int*)(base + oNa);

    std::vector<double> h_fn2(R), h_rn2(R), h_rel(R, 0.0);
    std::vector<int> h_act(R), h_frz(R), its(R, 0);

#define TRYC(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) return fail_cuda(_e); } while (0)
    // ---- the iterations of a cycle run as CUDA graphs, one per iteration index
    //      j, captured on first use and replayed on `st`; they are valid while
    //      the work space, the right-hand-side count, the tolerance and timing
    //      stay the same ----
    TRYC(sweep_prepare(h, R, st));
    if (!h->gm_graphs || h->gm_graph_R != R || h->gm_graph_buf != h->gm_buf || h->gm_graph_tol != tol ||
        h->gm_graph_timing != h->timing) {
        drop_graphs(h);
        GmGraph* G = new GmGraph[m];
        memset(G, 0, sizeof(GmGraph) * m);
        h->gm_graphs = G;
        h->gm_graph_R = R;
        h->gm_graph_buf = h->gm_buf;
        h->gm_graph_tol = tol;
        h->gm_graph_timing = h->timing;
    }
    if (!h->gm_cap_stream) {
        cudaStream_t cs_;
        TRYC(cudaStreamCreateWithFlags(&cs_, cudaStreamNonBlocking));
        h->gm_cap_stream = (void*)cs_;
    }
    GmGraph* G = static_cast<GmGraph*>(h->gm_graphs);
    // iteration j of a cycle: apply, matvec, CGS2, norm, Hessenberg column,
    // next basis vector, Givens rotation and the convergence test, captured
    // from stream q (timing events become event-record nodes of the graph)
    auto iteration = [&](int j, cudaStream_t q, cudaEvent_t* tev) -> cudaError_t {
        float2* Vj = V + (size_t)j * vs;
        float2* Zj = Z + (size_t)j * vs;
        cudaError_t e = cudaSuccess;
        if (tev) e = cudaEventRecordWithFlags(tev[0], q, cudaEventRecordExternal);
        if (e == cudaSuccess) e = launch_sweep(h, Vj, Zj, R, 0, 0, q);
        if (e == cudaSuccess && tev) e = cudaEventRecordWithFlags(tev[1], q, cudaEventRecordExternal);
        if (e == cudaSuccess) e = launch_stencil_c64(h, Zj, w, R, q);
        if (e == cudaSuccess && tev) e = cudaEventRecordWithFlags(tev[2], q, cudaEventRecordExternal);
        // classical Gram-Schmidt, twice (CGS2)
        double2* Hc = H + (size_t)j * (m + 1);
        if (e == cudaSuccess) e = gm_dots(h, V, vs, 0, j + 1, w, n3, R, part, Hc, m * (m + 1), 0, q);
        if (e == cudaSuccess) e = gm_axpy(h, V, vs, j + 1, Hc, m * (m + 1), w, n3, R, q);
        if (e == cudaSuccess) e = gm_dots(h, V, vs, 0, j + 1, w, n3, R, part, tmp, m + 1, 0, q);
        if (e == cudaSuccess) e = gm_axpy(h, V, vs, j + 1, tmp, m + 1, w, n3, R, q);
        if (e == cudaSuccess) e = gm_addcol(h, tmp, m + 1, Hc, m * (m + 1), j + 1, R, q);
        if (e == cudaSuccess) e = gm_norm2_c64(h, w, n3, R, part, wn2, q);
        if (e == cudaSuccess) e = gm_subdiag(h, wn2, H, inv, frozen, R, m, j, q);
        if (e == cudaSuccess) e = gm_scale_c64(h, w, inv, V + (size_t)(j + 1) * vs, n3, R, q);
        if (e == cudaSuccess) e = gm_givens(h, H, cs, sn, g, est, frozen, R, m, j, q);
        if (e == cudaSuccess) e = gm_converge(h, est, fn2, tol, maxit, frozen, its_d, mlen, j, R, nact_d, q);
        return e;
    };
    auto capture = [&](int j) -> cudaError_t {
        cudaStream_t q = (cudaStream_t)h->gm_cap_stream;
        if (h->timing)
            for (auto& ev : G[j].ev)
                if (!ev) {
                    cudaError_t e = cudaEventCreate(&ev);
                    if (e != cudaSuccess) return e;
                }
        const long long before = h->launches;
        cudaError_t e = cudaStreamBeginCapture(q, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaError_t e1 = iteration(j, q, h->timing ? G[j].ev : nullptr);
        cudaGraph_t gr = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(q, &gr);
        G[j].nlaunch = h->launches - before;      // counted again at every replay
        h->launches = before;
        if (e1 == cudaSuccess) e1 = e2;
        if (e1 == cudaSuccess) e1 = cudaGraphInstantiate(&G[j].exec, gr, 0);
        if (gr) cudaGraphDestroy(gr);
        return e1;
    };

    TRYC(gm_norm2_c64(h, f, n3, R, part, fn2, st));
    TRYC(cudaMemcpyAsync(h_fn2.data(), fn2, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    TRYC(cudaMemsetAsync(u64, 0, sizeof(double2) * (size_t)vs, st));
    TRYC(cudaMemsetAsync(its_d, 0, sizeof(int) * R, st));
    TRYC(cudaStreamSynchronize(st));

    int status = HELM_OK;
    for (;;) {
        // true residual in FP64 and the stopping test
        void* evr;
        helm_time_begin(h, st, &evr);
        TRYC(launch_residual_c128(h, f, u64, r64, R, st));
        helm_time_end(h, st, evr, 1, R);
        TRYC(gm_norm2_c128(h, r64, n3, R, part, rn2, st));
        TRYC(cudaMemcpyAsync(h_rn2.data(), rn2, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        TRYC(cudaStreamSynchronize(st));
        int nact = 0;
        for (int r = 0; r < R; ++r) {
            h_rel[r] = h_fn2[r] > 0.0 ? sqrt(h_rn2[r] / h_fn2[r]) : 0.0;
            if (!isfinite(h_rel[r])) {                 // a non-finite residual ends this right-hand side
                h_act[r] = 0;
                h_frz[r] = 1;
                continue;
            }
            h_act[r] = (h_fn2[r] > 0.0 && h_rel[r] > tol && its[r] < maxit) ? 1 : 0;
            h_frz[r] = !h_act[r];
            nact += h_act[r];
        }
        if (nact == 0) break;
        TRYC(cudaMemcpyAsync(active, h_act.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
        TRYC(cudaMemcpyAsync(frozen, h_frz.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
        TRYC(cudaMemsetAsync(mlen, 0, sizeof(int) * R, st));
        TRYC(gm_cycle_start(h, rn2, g, inv, active, R, m, st));
        TRYC(gm_scale_c128(h, r64, inv, V, n3, R, st));
        int jend = 0;
        for (int j = 0; j < m; ++j) {
            if (!G[j].exec) TRYC(capture(j));
            TRYC(cudaGraphLaunch(G[j].exec, st));
            h->launches += G[j].nlaunch;
            int left = 0;
            TRYC(cudaMemcpyAsync(&left, nact_d, sizeof(int), cudaMemcpyDeviceToHost, st));
            TRYC(cudaStreamSynchronize(st));
            if (h->timing) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, G[j].ev[0], G[j].ev[1]) == cudaSuccess) stats_add(h, 0, R, ms);
                if (cudaEventElapsedTime(&ms, G[j].ev[1], G[j].ev[2]) == cudaSuccess) stats_add(h, 1, R, ms);
                cudaGetLastError();          // a failed query must not surface at the next launch
            }
            jend = j + 1;
            if (left == 0) break;
        }
        TRYC(gm_cycle_len(h, active, mlen, jend, R, st));
        TRYC(gm_backsolve(h, H, g, y, mlen, R, m, st));
        TRYC(gm_update(h, Z, vs, y, m, mlen, u64, n3, R, st));
        TRYC(cudaMemcpyAsync(its.data(), its_d, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
        // the host vectors above must stay alive until the copies are done
        TRYC(cudaStreamSynchronize(st));
    }
    TRYC(gm_to_c64(h, u64, (float2*)u_, vs, st));
    int herr = 0;
    TRYC(cudaMemcpyAsync(&herr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRYC(cudaStreamSynchronize(st));
#undef TRYC
    for (int r = 0; r < R; ++r) {
        if (iters) iters[r] = its[r];
        if (relres) relres[r] = h_rel[r];
        if (!(h_rel[r] <= tol)) status = HELM_ENOCONV;   // also a non-finite residual
    }
    if (herr & 2) return HELM_ETIMEOUT;
    return status;
}

}  // extern "C"

extern "C" {

int helm_solve_adjoint(helm_handle h, const void* g, void* lam, int nrhs, double tol, int* iters,
                       double* relres, void* stream) {
    if (!h || !g || !lam || nrhs < 1 || !(tol > 0.0) || g == lam) return HELM_EINVAL;
    if (h->nsub) {
        if (nrhs != batch_total(h)) return HELM_EINVAL;
        size_t off = 0;
        int k = 0, rc = HELM_OK;
        for (int p = 0; p < h->nsub; ++p) {
            int q = helm_solve_adjoint(h->sub[p], (const float2*)g + off, (float2*)lam + off, h->sub_nrhs[p],
                                       tol, iters ? iters + k : nullptr, relres ? relres + k : nullptr, stream);
            if (q < 0) return q;
            if (q == HELM_ENOCONV) rc = q;
            off += (size_t)h->sub_nrhs[p] * sub_points(h->sub[p]);
            k += h->sub_nrhs[p];
        }
        return rc;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t need = (size_t)nrhs * h->g.N * h->g.N * h->g.N;
    if (need > h->adj_elems) {
        if (h->adj_buf) cudaFree(h->adj_buf);
        h->adj_buf = nullptr;
        h->adj_elems = 0;
        cudaError_t e = cudaMalloc(&h->adj_buf, need * sizeof(float2));
        if (e != cudaSuccess) return fail_cuda(e);
        h->adj_elems = need;
    }
    // D g into the caller's output, solve A mu = D g into the work buffer, lambda = D^{-1} mu
    cudaError_t e = launch_scale_D(h, (const float2*)g, (float2*)lam, nrhs, 0, st);
    if (e != cudaSuccess) return fail_cuda(e);
    int rc = helm_solve(h, lam, h->adj_buf, nrhs, tol, iters, relres, stream);
    if (rc != HELM_OK && rc != HELM_ENOCONV) return rc;
    e = launch_scale_D(h, h->adj_buf, (float2*)lam, nrhs, 1, st);
    if (e != cudaSuccess) return fail_cuda(e);
    return rc;
}

int helm_velocity_gradient(helm_handle h, const void* lam, const void* u, int nrhs, double* grad, void* stream) {
    if (h && h->nsub) {
        if (!lam || !u || !grad || nrhs != batch_total(h)) return HELM_EINVAL;
        size_t off = 0, goff = 0;
        for (int p = 0; p < h->nsub; ++p) {
            int rc = helm_velocity_gradient(h->sub[p], (const float2*)lam + off, (const float2*)u + off,
                                            h->sub_nrhs[p], grad + goff, stream);
            if (rc != HELM_OK) return rc;
            off += (size_t)h->sub_nrhs[p] * sub_points(h->sub[p]);
            goff += sub_points(h->sub[p]);
        }
        return HELM_OK;
    }
    if (!h || !lam || !u || !grad || nrhs < 1) return HELM_EINVAL;
    cudaError_t e = launch_velocity_gradient(h, (const float2*)lam, (const float2*)u, nrhs, grad,
                                             (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e);
    return HELM_OK;
}

}  // extern "C"

extern "C" {

int helm_apply_batch(const helm_handle* hs, const void* const* r, void* const* z, const int* nrhs, int nprob,
                     void* stream) {
    if (!hs || !r || !z || !nrhs || nprob < 1 || nprob > HELM_MAX_BATCH) return HELM_EINVAL;
    for (int p = 0; p < nprob; ++p)
        if (!hs[p] || hs[p]->nsub || !r[p] || !z[p] || nrhs[p] < 1 || r[p] == z[p]) return HELM_EINVAL;
    for (int p = 1; p < nprob; ++p)   // one kernel instance per stored-factor format
        if (hs[p]->opts.precision != hs[0]->opts.precision || hs[p]->dense != hs[0]->dense) return HELM_ENOTSUP;
    cudaError_t e = launch_sweep_batch(const_cast<helm_ctx* const*>(hs), (const float2* const*)r,
                                       (float2* const*)z, nrhs, nprob, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e);
    return HELM_OK;
}

int helm_solve_batch(const helm_handle* hs, const void* const* f, void* const* u, const int* nrhs, int nprob,
                     double tol, int* iters, double* relres, void* stream) {
    if (!hs || !f || !u || !nrhs || nprob < 1 || nprob > HELM_MAX_BATCH || !(tol > 0.0)) return HELM_EINVAL;
    int off[HELM_MAX_BATCH + 1] = {0};
    for (int p = 0; p < nprob; ++p) {
        if (!hs[p] || hs[p]->nsub || !f[p] || !u[p] || nrhs[p] < 1 || f[p] == u[p]) return HELM_EINVAL;
        off[p + 1] = off[p] + nrhs[p];
    }
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);     // inputs are ready
    if (e != cudaSuccess) return fail_cuda(e);
    bool any_dense = false;
    for (int p = 0; p < nprob; ++p) any_dense = any_dense || hs[p]->dense;
    if (any_dense) {
        // a dense apply spans the whole GPU (its clusters wait on one another), so
        // two of them must never share the GPU: the solves run one after another
        int rc = HELM_OK;
        for (int p = 0; p < nprob; ++p) {
            int q = helm_solve(hs[p], f[p], u[p], nrhs[p], tol, iters ? iters + off[p] : nullptr,
                               relres ? relres + off[p] : nullptr, stream);
            if (q < 0 && rc >= 0) rc = q;
            if (q == HELM_ENOCONV && rc == HELM_OK) rc = q;
        }
        return rc;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    int codes[HELM_MAX_BATCH];
    std::vector<std::thread> th;
    for (int p = 0; p < nprob; ++p) {
        th.emplace_back([&, p]() {
            cudaSetDevice(dev);
            cudaStream_t st;
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
                codes[p] = HELM_ECUDA;
                return;
            }
            codes[p] = helm_solve(hs[p], f[p], u[p], nrhs[p], tol, iters ? iters + off[p] : nullptr,
                                  relres ? relres + off[p] : nullptr, st);
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        });
    }
    for (auto& t : th) t.join();
    int rc = HELM_OK;
    for (int p = 0; p < nprob; ++p)
        if (codes[p] < 0 && rc >= 0) rc = codes[p];
    if (rc == HELM_OK)
        for (int p = 0; p < nprob; ++p)
            if (codes[p] == HELM_ENOCONV) rc = HELM_ENOCONV;
    return rc;
}

int helm_tune(const float* c, double omega, int n, int b, const helm_opts* base, const helm_candidate* cands,
              int ncand, const void* f, int nrhs, double tol, double setup_weight, helm_tune_result* results,
              int* best, void* stream) {
    if (!c || !cands || ncand < 1 || !f || nrhs < 1 || !(tol > 0.0) || !(setup_weight >= 0.0) || !best ||
        n < 1 || b < 1)
        return HELM_EINVAL;
    *best = -1;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)n + 2 * (size_t)b;
    void* u = nullptr;
    cudaError_t e = cudaMalloc(&u, (size_t)nrhs * N * N * N * sizeof(float2));
    if (e != cudaSuccess) return fail_cuda(e);
    cudaEvent_t ev[3];
    for (auto& x : ev) cudaEventCreate(&x);
    std::vector<int> its(nrhs);
    std::vector<double> rel(nrhs);
    double best_score = 0.0;
    int first_err = HELM_OK;
    for (int q = 0; q < ncand; ++q) {
        helm_tune_result r;
        memset(&r, 0, sizeof(r));
        r.cand = cands[q];
        helm_opts o;
        helm_default_opts(&o);
        if (base) o = *base;
        o.apply_form = cands[q].apply_form;
        o.precision = cands[q].precision;
        o.schedule = cands[q].schedule;
        o.b_aux = cands[q].b_aux;
        helm_handle h = nullptr;
        cudaEventRecord(ev[0], st);
        r.status = helm_setup(c, omega, n, b, cands[q].d, &o, stream, &h);
        cudaEventRecord(ev[1], st);
        if (r.status == HELM_OK) {
            r.stored_bytes = helm_factor_bytes(h);
            r.status = helm_solve(h, f, u, nrhs, tol, its.data(), rel.data(), stream);
            cudaEventRecord(ev[2], st);
            cudaEventSynchronize(ev[2]);
            float ms1 = 0.f, ms2 = 0.f;
            cudaEventElapsedTime(&ms1, ev[0], ev[1]);
            cudaEventElapsedTime(&ms2, ev[1], ev[2]);
            r.setup_ms = ms1;
            r.solve_ms = ms2;
            for (int k = 0; k < nrhs; ++k) {
                r.iters_max = std::max(r.iters_max, its[k]);
                r.relres_max = std::max(r.relres_max, rel[k]);
            }
            r.score = setup_weight * r.setup_ms + r.solve_ms;
            helm_destroy(h);
        }
        cudaStreamSynchronize(st);
        if (r.status == HELM_OK && (*best < 0 || r.score < best_score)) {
            *best = q;
            best_score = r.score;
        }
        if (r.status != HELM_OK && first_err == HELM_OK) first_err = r.status;
        if (results) results[q] = r;
    }
    for (auto& x : ev) cudaEventDestroy(x);
    cudaFree(u);
    return *best >= 0 ? HELM_OK : first_err;
}

int helm_autotune(helm_handle h, int nrhs, int* stages_out, void* stream) {
    if (!h || nrhs < 1) return HELM_EINVAL;
    if (h->nsub) {
        for (int p = 0; p < h->nsub; ++p) {
            int rc = helm_autotune(h->sub[p], h->sub_nrhs[p], p == 0 ? stages_out : nullptr, stream);
            if (rc != HELM_OK) return rc;
        }
        return HELM_OK;
    }
    if (h->dense) return HELM_ENOTSUP;
    cudaStream_t st = (cudaStream_t)stream;
    const int M = h->g.B / 2;
    int Lz = 0;
    {
        // the probe slab's window length
        int m = h->g.b + (M - 1) * h->g.d, e2 = std::min(m + h->g.d, h->g.N), lo = m - h->g.b_aux;
        Lz = (M == 0) ? h->g.b : e2 - std::max(lo, 0);
    }
    const size_t n = (size_t)nrhs * Lz * h->g.N * h->g.N;
    float2* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 2 * n * sizeof(float2));
    if (e != cudaSuccess) return fail_cuda(e);
    e = cudaMemsetAsync(buf, 0, 2 * n * sizeof(float2), st);
    const int keep_stages = h->sweep_stages;
    const size_t keep_smem = h->sweep_smem;
    int best = keep_stages;
    float best_ms = 1e30f;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int cand[5] = {2, 3, 4, 6, 8};
    for (int q = 0; q < 5 && e == cudaSuccess; ++q) {
        if (sweep_config_stages(h, cand[q]) != HELM_OK) continue;
        e = launch_sweep(h, buf, buf + n, nrhs, 1, M, st);              // warm
        if (e != cudaSuccess) break;
        cudaEventRecord(a, st);
        e = launch_sweep(h, buf, buf + n, nrhs, 1, M, st);
        cudaEventRecord(b, st);
        if (e != cudaSuccess) break;
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_ms) { best_ms = ms; best = cand[q]; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess || sweep_config_stages(h, best) != HELM_OK) {
        h->sweep_stages = keep_stages;
        h->sweep_smem = keep_smem;
        return e != cudaSuccess ? fail_cuda(e) : HELM_ECUDA;
    }
    if (stages_out) *stages_out = best;
    return HELM_OK;
}

}  // extern "C"
