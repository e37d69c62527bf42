// Serving loop with continuous batching (host C++ around the library's own
// entry points).
//
// One worker thread moves every request through two device stages, each on the
// stream of an internal context taken from a pool (each pool context has its
// own scratch, so requests in flight never share buffers):
//   stage 1: upload of the array geometry and the CSMs, DAS map and compressed
//            grid of every bin, download of the compressed sizes S_f;
//   stage 2: restriction of b, PSF matrix of every bin's kept points, one
//            Gauss-Seidel launch for all the request's bins, power maps,
//            download of the results.
// A request enters stage 1 when a pool slot is free and its stage-1 memory plus
// the least its stage 2 can need fit the HBM budget beside the requests in
// flight, and stage 2 when its matrices fit the budget and its solve's share of
// the SMs fits the free half-SM units (the library's plan of that solve: a CTA
// that fills an SM counts twice); so the cooperative solves in flight always
// fit on the device together.  A request that does not fit even alone runs
// when nothing else is in flight, and stage 2 is always granted when no other
// request is solving, so a small budget slows the loop but never stalls it.  Requests that arrive while others run are admitted as
// memory and slots free up, and their kernels overlap on the device.  Device
// memory comes from the stream-ordered allocator of each request's stream.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Job {
    uint64_t ticket = 0;
    damas_request req{};
    std::vector<double> mic, freqs;
    float *h_C = nullptr;  // pinned copy of the CSMs
    // results (pinned)
    float *h_x = nullptr;
    double *h_tot = nullptr;
    int *h_Sf = nullptr;
    int *h_status = nullptr;
    double t_submit = 0, t_admit = 0, t_solve = 0, t_done = 0;
    int status = DAMAS_EBUSY;
    int stage = 0;  // 0 queued, 1 stage 1 running, 2 waiting for stage 2, 3 stage 2 running, 4 done
    int slot = -1;
    size_t bytes1 = 0, bytes2 = 0;
    int units = 0;  // half-SM units its solve holds (solve_half_sm_units)
    std::vector<int> ctas_f;
    cudaEvent_t ev1 = nullptr, ev2 = nullptr;
    // device buffers
    double *d_mic = nullptr;
    float *d_C = nullptr, *d_b = nullptr, *d_xfull = nullptr;
    int32_t *d_idx = nullptr, *d_Sf = nullptr, *d_status = nullptr;
    double *d_tot = nullptr;
    std::vector<float *> d_A, d_g2, d_bs, d_x;
};

}  // namespace

struct ServeState {
    damas_serve_cfg cfg{};
    int device = 0, sm_count = 0;
    std::mutex mu;
    std::deque<Job *> queue;
    std::map<uint64_t, Job *> jobs;
    uint64_t next_ticket = 1;
    std::thread worker;
    std::atomic<bool> stopping{false};
    std::vector<damas_ctx *> pool;
    std::vector<cudaStream_t> streams;
    std::vector<Job *> running;
    size_t held_bytes = 0;
    int held_units = 0;
};

namespace {

damas_geom job_geom(const Job &j) {
    damas_geom g;
    g.M = j.req.M;
    g.mic_xyz_dev = j.d_mic;
    g.nx = j.req.nx;
    g.ny = j.req.ny;
    g.x0 = j.req.x0;
    g.y0 = j.req.y0;
    g.dx = j.req.dx;
    g.dy = j.req.dy;
    g.z = j.req.z;
    g.c = j.req.c;
    g.formulation = j.req.formulation;
    g.diag_removal = 0;
    return g;
}

size_t stage1_bytes(const damas_request &r) {
    const size_t S = (size_t)r.nx * r.ny, F = r.n_bins;
    return (size_t)r.M * 3 * 8 + F * r.M * r.M * 8 + F * S * 8 + F * 4 + 64;
}

// The least memory stage 2 can need, known before the compressed sizes: every
// bin keeps at least G^0 (Algorithm 1) and, with a keep fraction f, at least
// ceil(f S) points; a full-grid request keeps all S.  Same terms as plan_stage2.
size_t stage2_bytes_lower(const damas_request &r) {
    const size_t S = (size_t)r.nx * r.ny, F = r.n_bins;
    size_t n = S;
    if (r.wavelet.levels > 0) {
        const int J = r.wavelet.levels;
        n = (size_t)(((r.nx - 1) >> J) + 1) * (size_t)(((r.ny - 1) >> J) + 1);
        if (r.wavelet.eps_mode == DAMAS_EPS_KEEP_FRAC) n = std::max(n, (size_t)ceil(r.wavelet.eps * (double)S));
        n = std::min(n, S);
    }
    return S * F * 4 + F * 8 + 64 + F * (n * (size_t)damas_lda((int)n) * 4 + n * 16);
}

// Stage 1 on the job's stream: uploads, DAS maps, compressed grids, S_f download.
int launch_stage1(ServeState &st, Job &j) {
    damas_ctx *jc = st.pool[j.slot];
    cudaStream_t s = st.streams[j.slot];
    const damas_request &r = j.req;
    const size_t S = (size_t)r.nx * r.ny, F = r.n_bins;
    const bool compress = r.wavelet.levels > 0;
    if (cudaMallocAsync((void **)&j.d_mic, (size_t)r.M * 3 * 8, s) != cudaSuccess ||
        cudaMallocAsync((void **)&j.d_C, F * r.M * r.M * 8, s) != cudaSuccess ||
        cudaMallocAsync((void **)&j.d_b, F * S * 4, s) != cudaSuccess ||
        cudaMallocAsync((void **)&j.d_idx, F * S * 4, s) != cudaSuccess ||
        cudaMallocAsync((void **)&j.d_Sf, F * 4, s) != cudaSuccess)
        return DAMAS_ENOMEM;
    cudaMemcpyAsync(j.d_mic, j.mic.data(), (size_t)r.M * 3 * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(j.d_C, j.h_C, F * r.M * r.M * 8, cudaMemcpyHostToDevice, s);
    const damas_geom g = job_geom(j);
    for (size_t f = 0; f < F; ++f) {
        int rc = das_map(jc, &g, j.freqs[f], j.d_C + f * r.M * r.M * 2, j.d_b + f * S, s);
        if (rc) return rc;
        if (compress) {
            rc = wavelet_compress_grid(jc, j.d_b + f * S, r.nx, r.ny, &r.wavelet, j.d_idx + f * S, j.d_Sf + f, nullptr,
                                       nullptr, s);
            if (rc) return rc;
        }
    }
    if (compress)
        cudaMemcpyAsync(j.h_Sf, j.d_Sf, F * 4, cudaMemcpyDeviceToHost, s);
    else
        for (size_t f = 0; f < F; ++f) j.h_Sf[f] = (int)S;
    cudaEventRecord(j.ev1, s);
    return cudaGetLastError() == cudaSuccess ? DAMAS_OK : DAMAS_ECUDA;
}

// Memory stage 2 needs, from the compressed sizes, and the share of the SMs
// its solve holds: the library's own plan of that solve (form, CTAs per system,
// CTAs per SM), so a single-CTA solve, whose one CTA fills an SM, is charged the
// whole SM.
int plan_stage2(const ServeState &st, Job &j) {
    const damas_request &r = j.req;
    const size_t S = (size_t)r.nx * r.ny;
    const int rows = st.cfg.rows_per_cta > 0 ? st.cfg.rows_per_cta : 512;
    j.bytes2 = S * r.n_bins * 4 + (size_t)r.n_bins * 8 + 64;
    j.ctas_f.assign(r.n_bins, 1);
    std::vector<damas_system> sys(r.n_bins);
    for (int f = 0; f < r.n_bins; ++f) {
        const size_t n = (size_t)j.h_Sf[f];
        j.bytes2 += n * (size_t)damas_lda((int)n) * 4 + n * 16;
        const int nb = (int)((n + 31) / 32);
        j.ctas_f[f] = std::max(1, std::min(nb, (int)((n + rows - 1) / rows)));
        memset(&sys[f], 0, sizeof(damas_system));
        sys[f].a_dtype = DAMAS_F32;
        sys[f].S = (int)n;
        sys[f].lda = damas_lda((int)n);
        sys[f].iters = r.iters;
        sys[f].ctas = j.ctas_f[f];
    }
    return solve_half_sm_units(st.pool[j.slot], sys.data(), r.n_bins, &j.units);
}

// Stage 2 on the job's stream: PSF matrices, one solve for all bins, power maps, downloads.
int launch_stage2(ServeState &st, Job &j) {
    damas_ctx *jc = st.pool[j.slot];
    cudaStream_t s = st.streams[j.slot];
    const damas_request &r = j.req;
    const size_t S = (size_t)r.nx * r.ny, F = r.n_bins;
    const bool compress = r.wavelet.levels > 0;
    const damas_geom g = job_geom(j);
    j.d_A.assign(F, nullptr);
    j.d_g2.assign(F, nullptr);
    j.d_bs.assign(F, nullptr);
    j.d_x.assign(F, nullptr);
    if (cudaMallocAsync((void **)&j.d_xfull, F * S * 4, s) != cudaSuccess ||
        cudaMallocAsync((void **)&j.d_tot, F * 8, s) != cudaSuccess ||
        cudaMallocAsync((void **)&j.d_status, 4, s) != cudaSuccess)
        return DAMAS_ENOMEM;
    std::vector<damas_system> sys(F);
    for (size_t f = 0; f < F; ++f) {
        const int n = j.h_Sf[f];
        const int lda = damas_lda(n);
        if (cudaMallocAsync((void **)&j.d_A[f], (size_t)n * lda * 4, s) != cudaSuccess ||
            cudaMallocAsync((void **)&j.d_g2[f], (size_t)n * 4, s) != cudaSuccess ||
            cudaMallocAsync((void **)&j.d_bs[f], (size_t)n * 4, s) != cudaSuccess ||
            cudaMallocAsync((void **)&j.d_x[f], (size_t)n * 4, s) != cudaSuccess)
            return DAMAS_ENOMEM;
        const int32_t *idx = compress ? j.d_idx + f * S : nullptr;
        int rc;
        if (compress)
            rc = damas_gather(jc, j.d_b + f * S, idx, n, j.d_bs[f], s);
        else
            rc = cudaMemcpyAsync(j.d_bs[f], j.d_b + f * S, (size_t)n * 4, cudaMemcpyDeviceToDevice, s) == cudaSuccess
                     ? DAMAS_OK
                     : DAMAS_ECUDA;
        if (rc) return rc;
        rc = damas_build_psf(jc, &g, j.freqs[f], idx, n, DAMAS_F32, j.d_A[f], lda, j.d_g2[f], s);
        if (rc) return rc;
        damas_system &d = sys[f];
        memset(&d, 0, sizeof(d));
        d.A_dev = j.d_A[f];
        d.a_dtype = DAMAS_F32;
        d.lda = lda;
        d.S = n;
        d.b_dev = j.d_bs[f];
        d.x_dev = j.d_x[f];
        d.init = DAMAS_INIT_ZERO;
        d.iters = r.iters;
        d.ctas = j.ctas_f[f];
    }
    damas_solve_cfg cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.status_dev = j.d_status;
    int rc = damas_solve(jc, sys.data(), (int)F, &cfg, s);
    if (rc) return rc;
    for (size_t f = 0; f < F; ++f) {
        const int n = j.h_Sf[f];
        rc = damas_scatter_power(jc, j.d_x[f], compress ? j.d_idx + f * S : nullptr, j.d_g2[f], n, j.d_xfull + f * S,
                                 (int)S, j.d_tot + f, s);
        if (rc) return rc;
    }
    cudaMemcpyAsync(j.h_x, j.d_xfull, F * S * 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(j.h_tot, j.d_tot, F * 8, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(j.h_status, j.d_status, 4, cudaMemcpyDeviceToHost, s);
    cudaEventRecord(j.ev2, s);
    return cudaGetLastError() == cudaSuccess ? DAMAS_OK : DAMAS_ECUDA;
}

void free_device(ServeState &st, Job &j) {
    cudaStream_t s = st.streams[j.slot];
    for (void *p : {(void *)j.d_mic, (void *)j.d_C, (void *)j.d_b, (void *)j.d_idx, (void *)j.d_Sf,
                    (void *)j.d_xfull, (void *)j.d_tot, (void *)j.d_status})
        if (p) cudaFreeAsync(p, s);
    for (auto *v : {&j.d_A, &j.d_g2, &j.d_bs, &j.d_x})
        for (float *p : *v)
            if (p) cudaFreeAsync(p, s);
    j.d_A.clear();
    j.d_g2.clear();
    j.d_bs.clear();
    j.d_x.clear();
}

// A request ends (done or failed): free its device memory once its stream is
// idle, return its memory, CTAs and pool slot, and publish the status.
void complete(ServeState &st, Job &j, int status, std::vector<bool> &busy) {
    if (status != DAMAS_OK) {
        // let the failed request's work finish, and clear a build status it left
        // on the pool context so that the slot's next request starts clean
        cudaStreamSynchronize(st.streams[j.slot]);
        damas_check(st.pool[j.slot], st.streams[j.slot]);
    }
    free_device(st, j);
    std::lock_guard<std::mutex> lk(st.mu);
    st.held_bytes -= j.bytes1 + j.bytes2;
    st.held_units -= j.units;
    busy[j.slot] = false;
    j.status = status;
    j.stage = 4;
    j.t_done = now_s();
    st.running.erase(std::find(st.running.begin(), st.running.end(), &j));
}

void worker_loop(ServeState *stp) {
    ServeState &st = *stp;
    cudaSetDevice(st.device);
    const size_t budget = st.cfg.hbm_budget_bytes;
    const int slots = st.cfg.sm_slots;
    std::vector<bool> busy(st.pool.size(), false);
    for (;;) {
        bool progress = false;
        // admit queued requests to stage 1: a free pool slot and stage-1 memory
        for (;;) {
            Job *j = nullptr;
            {
                std::lock_guard<std::mutex> lk(st.mu);
                if (st.queue.empty()) break;
                int slot = -1;
                for (size_t i = 0; i < busy.size(); ++i)
                    if (!busy[i]) {
                        slot = (int)i;
                        break;
                    }
                if (slot < 0) break;
                Job *q = st.queue.front();
                const size_t b1 = stage1_bytes(q->req);
                // its stage 1 and the least its stage 2 can need must fit beside
                // what the requests in flight hold (a request runs alone when it
                // does not fit even so)
                if (st.held_bytes + b1 + stage2_bytes_lower(q->req) > budget && !st.running.empty()) break;
                st.queue.pop_front();
                q->slot = slot;
                q->bytes1 = b1;
                st.held_bytes += b1;
                busy[slot] = true;
                q->t_admit = now_s();
                q->stage = 1;
                st.running.push_back(q);
                j = q;
            }
            const int rc = launch_stage1(st, *j);
            if (rc) complete(st, *j, rc, busy);
            progress = true;
        }
        std::vector<Job *> run;
        {
            std::lock_guard<std::mutex> lk(st.mu);
            run = st.running;
        }
        for (Job *j : run) {
            if (j->stage == 1 && cudaEventQuery(j->ev1) == cudaSuccess) {
                const int rc = plan_stage2(st, *j);
                if (rc) {
                    j->bytes2 = 0;  // nothing of stage 2 was charged
                    j->units = 0;
                    complete(st, *j, rc, busy);
                    continue;
                }
                j->stage = 2;
                progress = true;
            }
            if (j->stage == 2) {
                // stage 2 needs its matrices within the budget and its solver's
                // share of the SMs within the free units (always granted when no
                // other request is in stage 2)
                bool go;
                {
                    std::lock_guard<std::mutex> lk(st.mu);
                    int in_stage2 = 0;
                    for (Job *o : st.running) in_stage2 += o->stage == 3 ? 1 : 0;
                    go = in_stage2 == 0 ||
                         (st.held_bytes + j->bytes2 <= budget && st.held_units + j->units <= slots);
                    if (go) {
                        st.held_bytes += j->bytes2;
                        st.held_units += j->units;
                        j->stage = 3;
                        j->t_solve = now_s();
                    }
                }
                if (go) {
                    const int rc = launch_stage2(st, *j);
                    if (rc) {
                        complete(st, *j, rc, busy);
                        continue;
                    }
                    progress = true;
                }
            }
            if (j->stage == 3 && cudaEventQuery(j->ev2) == cudaSuccess) {
                complete(st, *j, *j->h_status, busy);
                progress = true;
            }
        }
        {
            std::lock_guard<std::mutex> lk(st.mu);
            if (st.stopping && st.queue.empty() && st.running.empty()) break;
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    for (cudaStream_t q : st.streams) cudaStreamSynchronize(q);
}

}  // namespace

void serve_shutdown(damas_ctx *ctx);

extern "C" {

int damas_serve_start(damas_ctx *ctx, const damas_serve_cfg *cfg) {
    if (!ctx) return DAMAS_EINVAL;
    if (ctx->serve) return ctx_fail(ctx, DAMAS_EBUSY, "serving loop already running");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ctx_fail(ctx, DAMAS_ECUDA, "cudaSetDevice");
    ServeState *st = new ServeState();
    if (cfg) st->cfg = *cfg;
    // 32 requests in flight, two solver CTAs per SM and teams of 768 rows per CTA:
    // measured best for p99 latency and throughput on the mixed request stream
    // (against 8 in flight and 512 rows: p99 2.29 -> 1.50-1.57 s, 247 -> 354 bins/s)
    if (st->cfg.max_inflight <= 0) st->cfg.max_inflight = 32;
    if (st->cfg.sm_slots <= 0) st->cfg.sm_slots = 2 * ctx->sm_count;
    if (st->cfg.rows_per_cta <= 0) st->cfg.rows_per_cta = 768;
    if (st->cfg.hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        st->cfg.hbm_budget_bytes = fr / 2;
        if (ctx->hbm_budget) st->cfg.hbm_budget_bytes = ctx->hbm_budget;  // the context's own cap
    }
    st->device = ctx->device;
    st->sm_count = ctx->sm_count;
    for (int i = 0; i < st->cfg.max_inflight; ++i) {
        damas_ctx *jc = nullptr;
        cudaStream_t s = nullptr;
        if (damas_create(&jc, ctx->device) != DAMAS_OK || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) {
            if (jc) damas_destroy(jc);
            for (damas_ctx *p : st->pool) damas_destroy(p);
            for (cudaStream_t q : st->streams) cudaStreamDestroy(q);
            delete st;
            return ctx_fail(ctx, DAMAS_ECUDA, "could not create the serving pool");
        }
        st->pool.push_back(jc);
        st->streams.push_back(s);
    }
    ctx->serve = st;
    st->worker = std::thread(worker_loop, st);
    return DAMAS_OK;
}

int damas_serve_submit(damas_ctx *ctx, const damas_request *req, uint64_t *ticket) {
    if (!ctx || !req || !ticket) return DAMAS_EINVAL;
    ServeState *st = ctx->serve;
    if (!st || st->stopping) return ctx_fail(ctx, DAMAS_EBUSY, "serving loop is not running");
    const damas_request &r = *req;
    if (r.M < 1 || r.M > DAMAS_MAX_MICS || !r.mic_xyz || r.nx < 1 || r.ny < 1 || r.n_bins < 1 || !r.freqs || !r.C ||
        r.iters < 0 || !(r.c > 0) || r.formulation != DAMAS_FORM_E || r.wavelet.levels < 0 || r.wavelet.levels > 15 ||
        (long long)r.nx * r.ny > (1ll << 22))
        return ctx_fail(ctx, DAMAS_EINVAL, "invalid request");
    Job *j = new Job();
    j->req = r;
    j->mic.assign(r.mic_xyz, r.mic_xyz + (size_t)r.M * 3);
    j->freqs.assign(r.freqs, r.freqs + r.n_bins);
    const size_t S = (size_t)r.nx * r.ny, F = r.n_bins;
    const size_t cbytes = F * r.M * r.M * 8;
    if (cudaMallocHost((void **)&j->h_C, cbytes) != cudaSuccess ||
        cudaMallocHost((void **)&j->h_x, F * S * 4) != cudaSuccess ||
        cudaMallocHost((void **)&j->h_tot, F * 8) != cudaSuccess ||
        cudaMallocHost((void **)&j->h_Sf, F * 4) != cudaSuccess ||
        cudaMallocHost((void **)&j->h_status, 4) != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(ctx, DAMAS_ENOMEM, "pinned host memory for the request");
    }
    memcpy(j->h_C, r.C, cbytes);
    *j->h_status = 0;
    cudaEventCreateWithFlags(&j->ev1, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&j->ev2, cudaEventDisableTiming);
    j->req.mic_xyz = nullptr;
    j->req.freqs = nullptr;
    j->req.C = nullptr;
    j->t_submit = now_s();
    std::lock_guard<std::mutex> lk(st->mu);
    j->ticket = st->next_ticket++;
    st->jobs[j->ticket] = j;
    st->queue.push_back(j);
    *ticket = j->ticket;
    return DAMAS_OK;
}

int damas_serve_poll(damas_ctx *ctx, uint64_t ticket, damas_result *res) {
    if (!ctx || !res) return DAMAS_EINVAL;
    ServeState *st = ctx->serve;
    if (!st) return ctx_fail(ctx, DAMAS_ENOTFOUND, "serving loop is not running");
    std::lock_guard<std::mutex> lk(st->mu);
    auto it = st->jobs.find(ticket);
    if (it == st->jobs.end()) return ctx_fail(ctx, DAMAS_ENOTFOUND, "unknown ticket");
    const Job &j = *it->second;
    memset(res, 0, sizeof(*res));
    res->status = j.stage == 4 ? j.status : DAMAS_EBUSY;
    res->n_bins = j.req.n_bins;
    res->S = j.req.nx * j.req.ny;
    res->t_submit = j.t_submit;
    res->t_admit = j.t_admit;
    res->t_solve = j.t_solve;
    res->t_done = j.t_done;
    res->hbm_bytes = j.bytes1 + j.bytes2;
    res->sm_units = j.units;
    if (j.stage == 4) {
        res->x = j.h_x;
        res->total_power = j.h_tot;
        res->S_sub = j.h_Sf;
    }
    return DAMAS_OK;
}

int damas_serve_release(damas_ctx *ctx, uint64_t ticket) {
    if (!ctx) return DAMAS_EINVAL;
    ServeState *st = ctx->serve;
    if (!st) return ctx_fail(ctx, DAMAS_ENOTFOUND, "serving loop is not running");
    Job *j = nullptr;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        auto it = st->jobs.find(ticket);
        if (it == st->jobs.end()) return ctx_fail(ctx, DAMAS_ENOTFOUND, "unknown ticket");
        if (it->second->stage != 4) return ctx_fail(ctx, DAMAS_EBUSY, "request still in flight");
        j = it->second;
        st->jobs.erase(it);
    }
    cudaFreeHost(j->h_C);
    cudaFreeHost(j->h_x);
    cudaFreeHost(j->h_tot);
    cudaFreeHost(j->h_Sf);
    cudaFreeHost(j->h_status);
    cudaEventDestroy(j->ev1);
    cudaEventDestroy(j->ev2);
    delete j;
    return DAMAS_OK;
}

int damas_serve_stop(damas_ctx *ctx) {
    if (!ctx) return DAMAS_EINVAL;
    if (!ctx->serve) return DAMAS_OK;
    serve_shutdown(ctx);
    return DAMAS_OK;
}

}  // extern "C"

void serve_shutdown(damas_ctx *ctx) {
    ServeState *st = ctx->serve;
    if (!st) return;
    st->stopping = true;
    if (st->worker.joinable()) st->worker.join();
    std::vector<uint64_t> left;
    for (auto &kv : st->jobs) left.push_back(kv.first);
    for (uint64_t t : left) {
        Job *j = st->jobs[t];
        cudaFreeHost(j->h_C);
        cudaFreeHost(j->h_x);
        cudaFreeHost(j->h_tot);
        cudaFreeHost(j->h_Sf);
        cudaFreeHost(j->h_status);
        cudaEventDestroy(j->ev1);
        cudaEventDestroy(j->ev2);
        delete j;
    }
    for (damas_ctx *p : st->pool) damas_destroy(p);
    for (cudaStream_t s : st->streams) cudaStreamDestroy(s);
    ctx->serve = nullptr;
    delete st;
}
