// Request server: continuous batching of spectrum and ODF requests on one device.
//
// A worker thread owns the context while the server runs.  Submitted requests
// wait in a FIFO queue; the worker admits the oldest one as soon as a stream slot
// is free and its estimated device memory fits the HBM budget, so requests that
// arrive while others run are started without waiting for the running ones, and
// their kernels overlap on the device (CUDA streams per slot).  Each request's work
// is the same sequence of kernels as the direct entry points: populations, synthesis
// in chunks of rows (bounded scratch), then the formal solution or the ODF, and a copy
// of the result to a pinned staging buffer.  Completion is detected by polling a CUDA
// event (no blocking wait on the device); the result is copied to the caller's host
// buffer and the request's latency recorded.
//
// Small requests are kept from waiting behind large ones in two ways.  A spectrum
// request (tens of milliseconds) is enqueued whole on a stream of the device's highest
// priority; an ODF request (seconds of work in hundreds of chunks) is dispatched one
// chunk of rows at a time on a stream of the lowest priority, the next chunk when the
// previous one's event has completed.  So at most one chunk of an ODF request is queued
// on the device, and the block scheduler starts a spectrum's CTAs ahead of that chunk's
// queued ones (there is no preemption: running CTAs finish).
#include <math.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace mpsa {
namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    int64_t id = 0;
    int kind = 0;
    int status = 0;              // 0 queued, 1 running, 2 done, < 0 error code
    std::string err;
    // spectrum inputs (host copies)
    std::vector<double> m, T, P, mu;
    int comp = 0;
    mpsa_lgrid win{};
    float* I_out = nullptr;
    // ODF inputs (host copies)
    std::vector<int32_t> sel;
    mpsa_lgrid grid{};
    std::vector<int64_t> bounds;
    std::vector<double> widths, cw;
    double* odf_out = nullptr;
    float* kc_out = nullptr;
    int mean_kind = MPSA_MEAN_ARITH;
    // sizes
    int N = 0;
    size_t out_bytes = 0, kc_bytes = 0, est = 0;
    // runtime
    int slot = -1;
    cudaStream_t st = nullptr;   // the slot's stream of this request's priority
    // ODF requests: dispatched one chunk of rows at a time; device buffers kept across chunks
    int next_row = 0;
    int* dsel = nullptr;
    float *kap = nullptr, *kc = nullptr;
    int64_t* db = nullptr;
    double *dcw = nullptr, *dw = nullptr, *dout = nullptr;
    cudaEvent_t ev = nullptr;
    Clock::time_point t_submit, t_start, t_done;
};

struct Slot {
    cudaStream_t st_hi = nullptr, st_lo = nullptr;   // highest and lowest priority
    void* pinned = nullptr;
    size_t pinned_bytes = 0;
    Req* r = nullptr;
};

}  // namespace
}  // namespace mpsa

struct mpsa_server {
    mpsa_ctx* ctx = nullptr;
    size_t budget = 0, used = 0, peak = 0;
    int rows_per_chunk = 8;
    std::vector<mpsa::Slot> slots;
    std::deque<mpsa::Req*> queue;
    std::map<int64_t, mpsa::Req*> reqs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    int64_t next_id = 1, n_done = 0, n_failed = 0;
    std::string worker_error;
};

namespace mpsa {
namespace {

size_t synth_scratch_bytes(const mpsa_ctx* c, int rows, int N) {
    // per (row, line) prep arrays, buckets and the crossing-search list (~61 B), per-line
    // placement (12 B), tile ranges, per (row, prep block) class counts and window-length sums
    const size_t nT = (size_t)(N + kTile - 1) / kTile, nb = (size_t)(c->L + kPrepLines - 1) / kPrepLines;
    return (size_t)rows * c->L * 64 + (size_t)c->L * 12 + (size_t)rows * kNumClasses * (nT + 3) * 4 +
           (size_t)rows * nb * (kNumClasses * 4 + 8) + (1 << 20);
}

int launch_spectrum(mpsa_server* s, Req* r, Slot& sl) {
    mpsa_ctx* c = s->ctx;
    cudaStream_t st = r->st;
    const int D = (int)r->m.size(), N = r->N, n_mu = (int)r->mu.size(), ne = c->n_el;
    Scratch sc(st, s->ctx->pool);
    double *dT, *dP, *dab, *dpop;
    float *fm, *fT, *fmu, *kap, *kc, *Iout;
    int* dsel;
    int rc;
    if ((rc = sc.alloc(&dT, D)) || (rc = sc.alloc(&dP, D)) || (rc = sc.alloc(&dab, ne)) ||
        (rc = sc.alloc(&dpop, (size_t)D * pop_stride(ne))) || (rc = sc.alloc(&fm, D)) || (rc = sc.alloc(&fT, D)) ||
        (rc = sc.alloc(&fmu, n_mu)) || (rc = sc.alloc(&kap, (size_t)D * N)) || (rc = sc.alloc(&kc, D)) ||
        (rc = sc.alloc(&dsel, D)) || (rc = sc.alloc(&Iout, (size_t)n_mu * N)))
        return rc;
    std::vector<float> hm(D), hT(D), hmu(n_mu);
    std::vector<int> hsel(D);
    for (int d = 0; d < D; ++d) hm[d] = (float)r->m[d], hT[d] = (float)r->T[d], hsel[d] = d;
    for (int q = 0; q < n_mu; ++q) hmu[q] = (float)r->mu[q];
    const double* ab = c->h_abund.data() + (size_t)r->comp * ne;
    MPSA_CUDA_TRY(cudaMemcpyAsync(dT, r->T.data(), D * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(dP, r->P.data(), D * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(dab, ab, ne * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(fm, hm.data(), D * sizeof(float), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(fT, hT.data(), D * sizeof(float), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(fmu, hmu.data(), n_mu * sizeof(float), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(dsel, hsel.data(), D * sizeof(int), cudaMemcpyHostToDevice, st));
    if ((rc = populations_device(ne, c->d_el, dab, 1, D, dT, dP, dpop, st))) return rc;
    for (int off = 0; off < D; off += s->rows_per_chunk) {
        const int nrow = std::min(s->rows_per_chunk, D - off);
        if ((rc = synth_rows(c, dpop, nrow, dsel + off, r->win.lambda0_nm, r->win.R, N, kap + (size_t)off * N, kc + off,
                             nullptr, nullptr, st)))
            return rc;
    }
    if ((rc = formal_launch(D, N, kap, kc, nullptr, fm, fT, r->win.lambda0_nm, log1p(1.0 / r->win.R), n_mu, fmu, Iout,
                            st)))
        return rc;
    MPSA_CUDA_TRY(cudaMemcpyAsync(sl.pinned, Iout, r->out_bytes, cudaMemcpyDeviceToHost, st));
    return MPSA_OK;
}

// ODF requests run one chunk of rows per dispatch: launch_odf allocates the request's
// buffers and copies its inputs, odf_chunk enqueues the next chunk (synthesis + ODF) and,
// after the last, the copies to the staging buffer and the frees.  The worker dispatches the
// next chunk when the previous one's event has completed, so at most one chunk of a large
// request is queued on the device at any time and other requests' kernels interleave.
template <class T>
int pool_alloc(mpsa_server* s, T** p, size_t n, cudaStream_t st) {
    const cudaError_t e = cudaMallocFromPoolAsync((void**)p, (n ? n : 1) * sizeof(T), s->ctx->pool, st);
    return e == cudaSuccess ? MPSA_OK
                            : fail(e == cudaErrorMemoryAllocation ? MPSA_ENOMEM : MPSA_ECUDA,
                                   "mpsa_server: cudaMallocFromPoolAsync(%zu bytes): %s", n * sizeof(T),
                                   cudaGetErrorString(e));
}

void odf_free(Req* r) {
    void* ps[7] = {r->dsel, r->kap, r->kc, r->db, r->dcw, r->dw, r->dout};
    for (void* p : ps)
        if (p) cudaFreeAsync(p, r->st);
    r->dsel = nullptr, r->kap = r->kc = nullptr, r->db = nullptr, r->dcw = r->dw = r->dout = nullptr;
}

int launch_odf(mpsa_server* s, Req* r, Slot&) {
    cudaStream_t st = r->st;
    const int n_sel = (int)r->sel.size(), N = r->N, K = (int)r->bounds.size() - 1, ns = (int)r->widths.size();
    const int chunk = std::min(s->rows_per_chunk, n_sel);
    int rc;
    if ((rc = pool_alloc(s, &r->dsel, n_sel, st)) || (rc = pool_alloc(s, &r->kap, (size_t)chunk * N, st)) ||
        (rc = pool_alloc(s, &r->kc, n_sel, st)) || (rc = pool_alloc(s, &r->db, K + 1, st)) ||
        (rc = pool_alloc(s, &r->dcw, ns + 1, st)) || (rc = pool_alloc(s, &r->dw, ns, st)) ||
        (rc = pool_alloc(s, &r->dout, (size_t)n_sel * K * ns, st))) {
        odf_free(r);
        return rc;
    }
    MPSA_CUDA_TRY(cudaMemcpyAsync(r->dsel, r->sel.data(), n_sel * sizeof(int), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(r->db, r->bounds.data(), (K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(r->dcw, r->cw.data(), (ns + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(r->dw, r->widths.data(), ns * sizeof(double), cudaMemcpyHostToDevice, st));
    r->next_row = 0;
    return MPSA_OK;
}

int odf_chunk(mpsa_server* s, Req* r, Slot& sl) {
    mpsa_ctx* c = s->ctx;
    cudaStream_t st = r->st;
    const int n_sel = (int)r->sel.size(), N = r->N, K = (int)r->bounds.size() - 1, ns = (int)r->widths.size();
    const int off = r->next_row, nrow = std::min(std::min(s->rows_per_chunk, n_sel), n_sel - off);
    int rc;
    if ((rc = synth_rows(c, c->d_pop, nrow, r->dsel + off, r->grid.lambda0_nm, r->grid.R, N, r->kap, r->kc + off,
                         nullptr, nullptr, st)))
        return rc;
    if ((rc = odf_launch(r->kap, nrow, N, K, r->db, ns, r->dcw, r->dw, r->dout + (size_t)off * K * ns, r->mean_kind,
                         st)))
        return rc;
    r->next_row = off + nrow;
    if (r->next_row == n_sel) {
        MPSA_CUDA_TRY(cudaMemcpyAsync(sl.pinned, r->dout, r->out_bytes, cudaMemcpyDeviceToHost, st));
        MPSA_CUDA_TRY(cudaMemcpyAsync((char*)sl.pinned + r->out_bytes, r->kc, r->kc_bytes, cudaMemcpyDeviceToHost, st));
        odf_free(r);
    }
    return MPSA_OK;
}

int launch(mpsa_server* s, Req* r, Slot& sl) {
    const size_t need = r->out_bytes + r->kc_bytes;
    if (sl.pinned_bytes < need) {
        if (sl.pinned) cudaFreeHost(sl.pinned), sl.pinned = nullptr, sl.pinned_bytes = 0;
        MPSA_CUDA_TRY(cudaHostAlloc(&sl.pinned, need, cudaHostAllocDefault));
        sl.pinned_bytes = need;
    }
    r->st = r->kind == MPSA_REQ_SPECTRUM ? sl.st_hi : sl.st_lo;
    int rc = r->kind == MPSA_REQ_SPECTRUM ? launch_spectrum(s, r, sl) : launch_odf(s, r, sl);
    if (rc == MPSA_OK && r->kind != MPSA_REQ_SPECTRUM) rc = odf_chunk(s, r, sl);
    if (rc != MPSA_OK) {
        if (r->kind != MPSA_REQ_SPECTRUM) odf_free(r);
        return rc;
    }
    MPSA_CUDA_TRY(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming));
    MPSA_CUDA_TRY(cudaEventRecord(r->ev, r->st));
    return MPSA_OK;
}

// The next chunk of a running ODF request (its previous chunk has completed).
int continue_odf(mpsa_server* s, Req* r, Slot& sl) {
    int rc = odf_chunk(s, r, sl);
    if (rc != MPSA_OK) {
        odf_free(r);
        return rc;
    }
    MPSA_CUDA_TRY(cudaEventRecord(r->ev, r->st));
    return MPSA_OK;
}

void finish(mpsa_server* s, Req* r, Slot& sl, int status) {
    if (status == 2) {
        if (r->kind == MPSA_REQ_SPECTRUM) {
            memcpy(r->I_out, sl.pinned, r->out_bytes);
        } else {
            memcpy(r->odf_out, sl.pinned, r->out_bytes);
            if (r->kc_out) memcpy(r->kc_out, (char*)sl.pinned + r->out_bytes, r->kc_bytes);
        }
    }
    if (r->ev) cudaEventDestroy(r->ev), r->ev = nullptr;
    r->status = status;
    r->t_done = Clock::now();
    s->used -= r->est;
    sl.r = nullptr;
    if (status == 2) ++s->n_done; else ++s->n_failed;
}

void worker_loop(mpsa_server* s) {
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool running = false;
        for (auto& sl : s->slots) {
            if (!sl.r) continue;
            const cudaError_t q = cudaEventQuery(sl.r->ev);
            if (q == cudaSuccess && sl.r->kind != MPSA_REQ_SPECTRUM && sl.r->next_row < (int)sl.r->sel.size()) {
                Req* r = sl.r;
                lk.unlock();
                const int rc = continue_odf(s, r, sl);
                lk.lock();
                if (rc != MPSA_OK) {
                    r->err = mpsa_last_error();
                    cudaStreamSynchronize(r->st);
                    finish(s, r, sl, rc);
                } else {
                    running = true;
                }
            } else if (q == cudaSuccess) {
                finish(s, sl.r, sl, 2);
            } else if (q != cudaErrorNotReady) {
                cudaGetLastError();
                sl.r->err = cudaGetErrorString(q);
                finish(s, sl.r, sl, MPSA_ECUDA);
            } else {
                running = true;
            }
        }
        s->cv_done.notify_all();
        if (s->stop && s->queue.empty() && !running) break;
        // admission: oldest first, while a slot is free and the memory estimate fits
        while (!s->queue.empty()) {
            Req* r = s->queue.front();
            Slot* free_slot = nullptr;
            for (auto& sl : s->slots)
                if (!sl.r) { free_slot = &sl; break; }
            if (!free_slot) break;
            if (s->used + r->est > s->budget && running) break;
            s->queue.pop_front();
            s->used += r->est;
            if (s->used > s->peak) s->peak = s->used;
            free_slot->r = r;
            r->slot = (int)(free_slot - s->slots.data());
            r->status = 1;
            r->t_start = Clock::now();
            lk.unlock();
            const int rc = launch(s, r, *free_slot);
            lk.lock();
            if (rc != MPSA_OK) {
                r->err = mpsa_last_error();
                if (r->st) cudaStreamSynchronize(r->st);
                finish(s, r, *free_slot, rc);
                s->cv_done.notify_all();
            } else {
                running = true;
            }
        }
        if (running) s->cv_work.wait_for(lk, std::chrono::microseconds(200));
        else if (!s->stop) s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
    }
}

}  // namespace
}  // namespace mpsa

using namespace mpsa;

extern "C" {

int mpsa_server_create(mpsa_server** out, mpsa_ctx* ctx, size_t hbm_budget_bytes, int32_t max_inflight,
                       int32_t rows_per_chunk) {
    if (!out || !ctx) return fail(MPSA_EINVAL, "mpsa_server_create: NULL argument");
    if (max_inflight < 1 || max_inflight > 64) return fail(MPSA_EINVAL, "mpsa_server_create: max_inflight %d", max_inflight);
    if (rows_per_chunk < 1) rows_per_chunk = 8;
    if (rows_per_chunk > 65535) rows_per_chunk = 65535;   // rows of one ODF launch
    if (ctx->L < 1 || !ctx->d_pop) return fail(MPSA_ESTATE, "mpsa_server_create: load a line list and a grid first");
    MPSA_CUDA_TRY(cudaSetDevice(ctx->device));
    mpsa_server* s = new mpsa_server();
    s->ctx = ctx;
    s->budget = hbm_budget_bytes;
    s->rows_per_chunk = rows_per_chunk;
    s->slots.resize(max_inflight);
    int least = 0, greatest = 0;
    MPSA_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    for (auto& sl : s->slots) {
        cudaError_t e = cudaStreamCreateWithPriority(&sl.st_hi, cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.st_lo, cudaStreamNonBlocking, least);
        if (e != cudaSuccess) {
            for (auto& q : s->slots) {
                if (q.st_hi) cudaStreamDestroy(q.st_hi);
                if (q.st_lo) cudaStreamDestroy(q.st_lo);
            }
            delete s;
            return fail(MPSA_ECUDA, "mpsa_server_create: %s", cudaGetErrorString(e));
        }
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return MPSA_OK;
}

int mpsa_server_submit(mpsa_server* s, const mpsa_request* q, int64_t* ticket) {
    if (!s || !q || !ticket) return fail(MPSA_EINVAL, "mpsa_server_submit: NULL argument");
    mpsa_ctx* c = s->ctx;
    Req* r = new Req();
    r->kind = q->kind;
    int rc;
    if (q->kind == MPSA_REQ_SPECTRUM) {
        const int D = q->atm.n_depth;
        if (D < 2 || D > 256 || !q->atm.m || !q->atm.T || !q->atm.P || !q->mu || q->n_mu < 1 || q->n_mu > 16 || !q->I_out) {
            delete r;
            return fail(MPSA_EINVAL, "mpsa_server_submit: bad spectrum request");
        }
        if (q->atm.comp < 0 || q->atm.comp >= c->n_comp) {
            delete r;
            return fail(MPSA_EINVAL, "mpsa_server_submit: comp %d", q->atm.comp);
        }
        for (int d = 0; d < D; ++d)
            if (!(q->atm.m[d] > 0) || !(q->atm.T[d] > 0) || !(q->atm.P[d] > 0) || (d > 0 && !(q->atm.m[d] > q->atm.m[d - 1]))) {
                delete r;
                return fail(MPSA_EINVAL, "mpsa_server_submit: bad atmosphere at depth %d", d);
            }
        for (int k = 0; k < q->n_mu; ++k)
            if (!(q->mu[k] > 0 && q->mu[k] <= 1)) {
                delete r;
                return fail(MPSA_EINVAL, "mpsa_server_submit: mu[%d]", k);
            }
        if ((rc = check_grid(&q->win, &r->N))) { delete r; return rc; }
        r->m.assign(q->atm.m, q->atm.m + D);
        r->T.assign(q->atm.T, q->atm.T + D);
        r->P.assign(q->atm.P, q->atm.P + D);
        r->mu.assign(q->mu, q->mu + q->n_mu);
        r->comp = q->atm.comp;
        r->win = q->win;
        r->I_out = q->I_out;
        r->out_bytes = (size_t)q->n_mu * r->N * sizeof(float);
        r->est = (size_t)D * r->N * 4 + (size_t)q->n_mu * r->N * 4 + synth_scratch_bytes(c, std::min(s->rows_per_chunk, D), r->N);
    } else if (q->kind == MPSA_REQ_ODF) {
        if (q->n_sel < 1 || !q->sel || !q->bounds || !q->widths || !q->odf_out || q->K < 1 || q->n_steps < 1 || q->n_steps > 32) {
            delete r;
            return fail(MPSA_EINVAL, "mpsa_server_submit: bad ODF request");
        }
        const int rows = c->n_comp * c->n_points;
        for (int i = 0; i < q->n_sel; ++i)
            if (q->sel[i] < 0 || q->sel[i] >= rows) {
                delete r;
                return fail(MPSA_EINVAL, "mpsa_server_submit: sel[%d] = %d", i, q->sel[i]);
            }
        if ((rc = check_grid(&q->grid, &r->N))) { delete r; return rc; }
        r->cw.resize(q->n_steps + 1);
        // the ODF runs in launches of at most rows_per_chunk rows
        if ((rc = odf_check("mpsa_server_submit", std::min(q->n_sel, s->rows_per_chunk), r->N, q->K, q->bounds,
                            q->n_steps, q->widths, q->mean_kind, r->cw.data()))) {
            delete r;
            return rc;
        }
        r->sel.assign(q->sel, q->sel + q->n_sel);
        r->grid = q->grid;
        r->mean_kind = q->mean_kind;
        r->bounds.assign(q->bounds, q->bounds + q->K + 1);
        r->widths.assign(q->widths, q->widths + q->n_steps);
        r->odf_out = q->odf_out;
        r->kc_out = q->kappa_c_out;
        r->out_bytes = (size_t)q->n_sel * q->K * q->n_steps * sizeof(double);
        r->kc_bytes = (size_t)q->n_sel * sizeof(float);
        const int chunk = std::min(s->rows_per_chunk, q->n_sel);
        r->est = (size_t)chunk * r->N * 4 + r->out_bytes + synth_scratch_bytes(c, chunk, r->N);
    } else {
        delete r;
        return fail(MPSA_EINVAL, "mpsa_server_submit: kind %d", q->kind);
    }
    if (r->est > s->budget) {
        const size_t est = r->est;
        delete r;
        return fail(MPSA_ENOMEM, "mpsa_server_submit: request needs about %zu bytes, budget is %zu", est, s->budget);
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return fail(MPSA_ESTATE, "mpsa_server_submit: server is stopping");
        }
        r->id = s->next_id++;
        r->t_submit = Clock::now();
        s->reqs[r->id] = r;
        s->queue.push_back(r);
        *ticket = r->id;
    }
    s->cv_work.notify_one();
    return MPSA_OK;
}

int mpsa_server_wait(mpsa_server* s, int64_t ticket, int32_t timeout_ms, double* latency_ms) {
    if (!s) return fail(MPSA_EINVAL, "mpsa_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(MPSA_EINVAL, "mpsa_server_wait: unknown ticket %lld", (long long)ticket);
    Req* r = it->second;
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                        [&] { return r->status == 2 || r->status < 0; });
    if (!ok) return fail(MPSA_ETIMEOUT, "mpsa_server_wait: ticket %lld not done after %d ms", (long long)ticket, timeout_ms);
    const int st = r->status;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    std::string err = r->err;
    s->reqs.erase(it);
    delete r;
    if (st < 0) return fail(st, "mpsa_server_wait: request failed: %s", err.c_str());
    return MPSA_OK;
}

int mpsa_server_get_stats(mpsa_server* s, mpsa_server_stats* out) {
    if (!s || !out) return fail(MPSA_EINVAL, "mpsa_server_get_stats: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->completed = s->n_done;
    out->failed = s->n_failed;
    out->queued = (int64_t)s->queue.size();
    int64_t running = 0;
    for (auto& sl : s->slots)
        if (sl.r) ++running;
    out->running = running;
    out->bytes_in_use = s->used;
    out->bytes_peak = s->peak;
    out->submitted = s->next_id - 1;
    return MPSA_OK;
}

int mpsa_server_cancel_queued(mpsa_server* s, int64_t* n_cancelled) {
    if (!s) return fail(MPSA_EINVAL, "mpsa_server_cancel_queued: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    int64_t n = 0;
    for (Req* r : s->queue) {
        r->status = MPSA_ESTATE;
        r->err = "cancelled before admission";
        r->t_done = Clock::now();
        ++n;
    }
    s->queue.clear();
    s->n_failed += n;
    if (n_cancelled) *n_cancelled = n;
    s->cv_done.notify_all();
    return MPSA_OK;
}

void mpsa_server_destroy(mpsa_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto& sl : s->slots) {
        if (sl.st_hi) cudaStreamSynchronize(sl.st_hi), cudaStreamDestroy(sl.st_hi);
        if (sl.st_lo) cudaStreamSynchronize(sl.st_lo), cudaStreamDestroy(sl.st_lo);
        if (sl.pinned) cudaFreeHost(sl.pinned);
    }
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
}

}  // extern "C"
