// bls_server.cpp -- serving: bls_submit / bls_poll with continuous batching.
//
// One scheduler thread per plan owns a CUDA stream and a table of device slots.  Each step
//   1. retires cancelled requests and admits queued ones (first come, first served) while
//      a slot is free and their device memory fits the plan's budget; admission copies the
//      curve to the device and runs the prep kernel for it;
//   2. gives every active request its share of a fixed amount of work (point x frequency
//      units, box evaluations counted at their relative cost) as its next frequency tiles,
//      and runs all of them in one persistent fold-bin-sweep launch per block-size class;
//   3. reduces the requests whose last tile ran and copies their peaks back.
// Steps are pipelined two deep: after enqueueing step k the thread waits for step k-1 and
// retires its finished requests (results, memory), so the GPU works on step k while the
// host finishes k-1 and prepares k+1.  Admission copies run on a copy stream (the curve
// arrays are pageable) that the compute stream waits for.  Requests that arrive while
// others are on the GPU join at the next step, so their work overlaps on the device
// (iteration-level continuous batching); no kernel waits on the host.  The per-frequency
// arithmetic is the batched search's, so a request's result is the same alone and in a mix.
//
// Plans of the other algorithms (the plain FP64 baseline, the unbinned search) are served
// sequentially through the same queue: the scheduler takes the oldest request, runs it as
// one search of one curve, and retires it before taking the next -- first come, first
// served, no batching, which is how a one-curve-per-launch code serves a stream.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>

#include "bls_plan.h"

using namespace blsgpu;

namespace blsgpu {

namespace {

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Relative cost of one box evaluation against one point x frequency unit (measured ratio
// of the two loops of the fold-bin-sweep kernel on B300).
constexpr double kEvalCost = 0.3;

enum class RState { Queued, Active, Done, Failed, Cancelled };

struct Request {
    uint64_t id = 0;
    std::vector<double> t, freqs;
    std::vector<float> y, dy;
    CurveSpec spec{};
    bls_curve src{};              // the submitted descriptor, pointing at the copies above
    FoldGeom geom{};
    size_t bytes = 0;
    void* dmem = nullptr;
    int slot = -1;
    long long ntiles = 0, next_tile = 0;
    double tile_cost = 0.0;
    RState state = RState::Queued;
    bool cancel = false;
    bool finishing = false;       // its last tiles are in the step in flight
    bls_status status = BLS_OK;
    std::string error;
    std::vector<bls_peak> peaks;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
};

}  // namespace

struct Server {
    bls_plan_impl* P = nullptr;
    int max_active = 64;
    double step_units = 2.0e9;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<Request*> queue;
    std::vector<Request*> slots;          // active requests by slot
    std::unordered_map<uint64_t, Request*> all;
    uint64_t next_id = 1;
    cudaStream_t stream = nullptr;
    size_t in_use = 0, peak_use = 0;
    uint64_t submitted = 0, completed = 0, cancelled = 0, failed = 0, steps = 0;
    std::vector<double> latencies;
    long fail_every = 0, alloc_count = 0;   // test hook: simulated allocation failures
    std::string fatal;                       // set when the device became unusable

    DevBuf cdesc, ranges, prefix, counter, err, dslots, dpeaks;
    HostBuf h_cdesc;
    // host staging of a step, one set per pipeline parity
    struct StepBufs { HostBuf h_ranges, h_prefix, h_slots, h_peaks, h_err; } sb[2];
    cudaEvent_t ev_step[2] = {};
    int parity = 0;
    // the step in flight
    bool inflight = false;
    int fl_parity = 0;
    std::vector<Request*> fl_finishing;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copy = nullptr;
    // requests of different block sizes run in different fold-sweep launches; these
    // streams let the launches of one step share the GPU instead of queueing behind each
    // other (each forks from and joins back into `stream`)
    static constexpr int kClassStreams = 4;
    cudaStream_t cls_stream[kClassStreams] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kClassStreams] = {};

    void run();
    bool step();
    bool step_sequential();
    bool retire_inflight();
    void fail_all(const std::string& why);
};

void Server::fail_all(const std::string& why)
{
    std::lock_guard<std::mutex> lk(mu);
    fatal = why;
    for (Request* r : slots)
        if (r) { r->state = RState::Failed; r->status = BLS_ERR_CUDA; r->error = why; ++failed; }
    std::fill(slots.begin(), slots.end(), nullptr);
    for (Request* r : queue) { r->state = RState::Failed; r->status = BLS_ERR_CUDA; r->error = why; ++failed; }
    queue.clear();
    cv_done.notify_all();
}

void Server::run()
{
    cudaSetDevice(P->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] {
                if (stop) return true;
                if (inflight || !queue.empty()) return true;
                for (Request* r : slots) if (r) return true;
                return false;
            });
            if (stop) return;
        }
        if (!step()) return;
    }
}

// One request of a sequentially served plan: the oldest queued one, searched alone.
bool Server::step_sequential()
{
    Request* r = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (queue.empty()) return true;
        r = queue.front();
        queue.pop_front();
        r->state = RState::Active;
        r->t_admit = now_ms();
    }
    std::vector<bls_peak> pk((size_t)P->d.topk);
    const bls_status st = search_one_locked(P, &r->src, pk.data());
    const std::string why = st == BLS_OK ? std::string() : std::string(bls_last_error());
    std::lock_guard<std::mutex> lk(mu);
    if (r->cancel) {
        r->state = RState::Cancelled;
        r->status = BLS_ERR_CANCELLED;
        ++cancelled;
    } else if (st == BLS_OK) {
        r->peaks = std::move(pk);
        r->state = RState::Done;
        r->status = BLS_OK;
        ++completed;
    } else {
        r->state = RState::Failed;
        r->status = st;
        r->error = why;
        ++failed;
    }
    r->t_done = now_ms();
    latencies.push_back(r->t_done - r->t_submit);
    ++steps;
    r->t.clear(); r->t.shrink_to_fit();
    r->y.clear(); r->y.shrink_to_fit();
    r->dy.clear(); r->dy.shrink_to_fit();
    r->freqs.clear(); r->freqs.shrink_to_fit();
    cv_done.notify_all();
    return true;
}

// One scheduler step; returns false when the device failed.
bool Server::step()
{
    NvtxRange r_step("bls.server.step");
    if (P->d.algo != BLS_ALGO_TILED) return step_sequential();
    cudaError_t e;
    std::vector<Request*> admitted, retire_cancel;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (int s = 0; s < max_active; ++s) {
            Request* r = slots[s];
            if (r && r->cancel && !r->finishing) { retire_cancel.push_back(r); slots[s] = nullptr; }
        }
        // admission: first come, first served, while a slot is free and memory fits
        while (!queue.empty()) {
            Request* r = queue.front();
            int free_slot = -1;
            for (int s = 0; s < max_active; ++s) if (!slots[s]) { free_slot = s; break; }
            if (free_slot < 0 || in_use + r->bytes > P->budget) break;
            queue.pop_front();
            ++alloc_count;
            if (fail_every > 0 && alloc_count % fail_every == 0) {
                r->state = RState::Failed;
                r->status = BLS_ERR_NOMEM;
                r->error = "device allocation failed (simulated)";
                ++failed;
                cv_done.notify_all();
                continue;
            }
            r->slot = free_slot;
            r->state = RState::Active;
            slots[free_slot] = r;
            in_use += r->bytes;
            peak_use = std::max(peak_use, in_use);
            admitted.push_back(r);
        }
    }
    for (Request* r : retire_cancel) {
        if (r->dmem) cudaFreeAsync(r->dmem, stream);
        std::lock_guard<std::mutex> lk(mu);
        in_use -= r->bytes;
        r->dmem = nullptr;
        r->state = RState::Cancelled;
        r->status = BLS_ERR_CANCELLED;
        ++cancelled;
        cv_done.notify_all();
    }

    // ---- admit: device memory, input copies, descriptors, prep
    const int par = parity;
    parity ^= 1;
    StepBufs& B = sb[par];
    CurveDesc* hd = h_cdesc.as<CurveDesc>();
    int* hs = B.h_slots.as<int>();
    int nadm = 0;
    for (Request* r : admitted) {
        e = cudaMallocAsync(&r->dmem, r->bytes, copy_stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            std::lock_guard<std::mutex> lk(mu);
            slots[r->slot] = nullptr;
            in_use -= r->bytes;
            r->dmem = nullptr;
            r->state = RState::Failed;
            r->status = BLS_ERR_NOMEM;
            r->error = std::string("device allocation failed: ") + cudaGetErrorString(e);
            ++failed;
            cv_done.notify_all();
            continue;
        }
        const CurveSpec& s = r->spec;
        char* base = static_cast<char*>(r->dmem);
        const long long n2 = (s.n + 1) & ~1;
        size_t off = 0;
        auto carve = [&](size_t bytes) { char* p = base + off; off += up256(bytes); return p; };
        double* dt_raw = reinterpret_cast<double*>(carve((size_t)s.n * 8));
        float* dy_raw = reinterpret_cast<float*>(carve((size_t)s.n * 4));
        float* ddy = s.dy ? reinterpret_cast<float*>(carve((size_t)s.n * 4)) : nullptr;
        double* dfr = s.freqs ? reinterpret_cast<double*>(carve((size_t)s.nf * 8)) : nullptr;
        float4* dpts = reinterpret_cast<float4*>(carve((size_t)(n2 + 2) * 16));
        double* ddt = reinterpret_cast<double*>(carve((size_t)(n2 + 2) * 8));
        float* dres = reinterpret_cast<float*>(carve((size_t)s.nf * 4));
        cudaMemcpyAsync(dt_raw, r->t.data(), (size_t)s.n * 8, cudaMemcpyHostToDevice, copy_stream);
        cudaMemcpyAsync(dy_raw, r->y.data(), (size_t)s.n * 4, cudaMemcpyHostToDevice, copy_stream);
        if (ddy) cudaMemcpyAsync(ddy, r->dy.data(), (size_t)s.n * 4, cudaMemcpyHostToDevice, copy_stream);
        if (dfr) cudaMemcpyAsync(dfr, r->freqs.data(), (size_t)s.nf * 8, cudaMemcpyHostToDevice, copy_stream);
        CurveDesc d;
        memset(&d, 0, sizeof(d));
        d.t = dt_raw; d.y = dy_raw; d.dy = ddy; d.freqs = dfr;
        d.pts = dpts; d.dt64 = ddt; d.res = dres;
        d.fmin = s.fmin; d.df = s.df;
        d.n = s.n; d.nf = s.nf; d.nb = s.nb; d.kmin = s.kmin; d.kmax = s.kmax; d.T = r->geom.T;
        hd[r->slot] = d;
        cudaMemcpyAsync(cdesc.as<CurveDesc>() + r->slot, &hd[r->slot], sizeof(CurveDesc),
                        cudaMemcpyHostToDevice, copy_stream);
        hs[nadm++] = r->slot;
        r->t_admit = now_ms();
    }
    int* dsl = dslots.as<int>();
    bool enq = false;   // anything enqueued in this step
    if (nadm > 0) {
        cudaEventRecord(ev_copy, copy_stream);
        cudaStreamWaitEvent(stream, ev_copy, 0);
        cudaMemsetAsync(err.p, 0, sizeof(int), stream);
        enq = true;
        cudaMemcpyAsync(dsl, hs, sizeof(int) * nadm, cudaMemcpyHostToDevice, stream);
        if ((e = launch_prep(cdesc.as<CurveDesc>(), dsl, nadm, err.as<int>(), P->d.phase, P->d.sum, stream)) != cudaSuccess) {
            fail_all(std::string("prep launch: ") + cudaGetErrorString(e));
            return false;
        }
    }

    // ---- this step's tiles: an equal share of the step's work per active request
    std::vector<Request*> act;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (Request* r : slots) if (r && r->dmem) act.push_back(r);
    }
    std::sort(act.begin(), act.end(), [](const Request* a, const Request* b) { return a->id < b->id; });
    std::vector<FoldGeom> geoms;
    std::vector<std::vector<std::pair<Request*, long long>>> cls;   // (request, tiles) per class
    const double share = act.empty() ? 0.0 : step_units / (double)act.size();
    std::vector<Request*> finishing;
    for (Request* r : act) {
        long long want = (long long)std::max(1.0, std::floor(share / r->tile_cost));
        long long take = std::min(want, r->ntiles - r->next_tile);
        if (take <= 0) continue;
        int k = -1;
        for (size_t q = 0; q < geoms.size(); ++q)
            if (geoms[q].T == r->geom.T && geoms[q].stride == r->geom.stride && geoms[q].chunk == r->geom.chunk &&
                geoms[q].ws == r->geom.ws) { k = (int)q; break; }
        if (k < 0) { geoms.push_back(r->geom); cls.emplace_back(); k = (int)geoms.size() - 1; }
        else geoms[k].smem = std::max(geoms[k].smem, r->geom.smem);
        cls[k].push_back({r, take});
        if (r->next_tile + take == r->ntiles) { finishing.push_back(r); r->finishing = true; }
    }
    TileRange* hr = B.h_ranges.as<TileRange>();
    long long* hp = B.h_prefix.as<long long>();
    size_t rr = 0, pp = 0;
    std::vector<size_t> r0(cls.size()), p0(cls.size());
    std::vector<long long> tot(cls.size());
    for (size_t q = 0; q < cls.size(); ++q) {
        r0[q] = rr;
        p0[q] = pp;
        long long acc = 0;
        for (auto& it : cls[q]) {
            hr[rr++] = TileRange{it.first->slot, (int)it.first->next_tile};
            hp[pp++] = acc;
            acc += it.second;
            it.first->next_tile += it.second;
        }
        hp[pp++] = acc;
        tot[q] = acc;
    }
    if (rr > 0) {
        if (!enq) { cudaMemsetAsync(err.p, 0, sizeof(int), stream); enq = true; }
        cudaMemcpyAsync(ranges.p, hr, rr * sizeof(TileRange), cudaMemcpyHostToDevice, stream);
        cudaMemcpyAsync(prefix.p, hp, pp * sizeof(long long), cudaMemcpyHostToDevice, stream);
        cudaMemsetAsync(counter.p, 0, cls.size() * sizeof(int), stream);
        const int nstr = (int)std::min<size_t>(cls.size(), (size_t)kClassStreams);
        if (nstr > 1) {
            cudaEventRecord(ev_fork, stream);
            for (int q = 0; q < nstr; ++q) cudaStreamWaitEvent(cls_stream[q], ev_fork, 0);
        }
        for (size_t q = 0; q < cls.size(); ++q) {
            FoldParams fp;
            fp.curves = cdesc.as<CurveDesc>();
            fp.ranges = ranges.as<TileRange>() + r0[q];
            fp.prefix = prefix.as<long long>() + p0[q];
            fp.nranges = (int)cls[q].size();
            fp.total = tot[q];
            fp.counter = counter.as<int>() + q;
            fp.err = err.as<int>();
            fp.chunk = geoms[q].chunk;
            fp.stride = geoms[q].stride;
            fp.wait_ns = handoff_limit_ns();
            const int bps = fold_blocks_per_sm(geoms[q].T, geoms[q].smem, P->d.phase,
                                               P->d.sum, P->d.sign, geoms[q].ws);
            long long grid = std::min<long long>((long long)P->sm_count * bps, tot[q]);
            cudaStream_t sq = nstr > 1 ? cls_stream[q % nstr] : stream;
            if ((e = launch_fold_sweep(fp, geoms[q].T, (int)std::max<long long>(grid, 1), P->d.phase,
                                       P->d.sum, geoms[q].ws, P->d.sign, geoms[q].smem,
                                       sq)) != cudaSuccess) {
                fail_all(std::string("fold-sweep launch: ") + cudaGetErrorString(e));
                return false;
            }
        }
        if (nstr > 1) {
            for (int q = 0; q < nstr; ++q) {
                cudaEventRecord(ev_join[q], cls_stream[q]);
                cudaStreamWaitEvent(stream, ev_join[q], 0);
            }
        }
    }
    // ---- reduce the requests whose last tile ran
    const int topk = P->d.topk;
    if (!finishing.empty()) {
        int nf = 0;
        int nbmax = 2;
        for (Request* r : finishing) { hs[nadm + nf++] = r->slot; nbmax = std::max(nbmax, r->spec.nb); }
        cudaMemcpyAsync(dsl + nadm, hs + nadm, sizeof(int) * nf, cudaMemcpyHostToDevice, stream);
        ReduceParams rp;
        rp.curves = cdesc.as<CurveDesc>();
        rp.slots = dsl + nadm;
        rp.peaks = dpeaks.as<DevPeak>();
        rp.spectrum = nullptr;
        rp.topk = topk;
        rp.sign = P->d.sign;
        rp.phase = P->d.phase;
        rp.sums = P->d.sum;
        rp.smem_bytes = reduce_smem_bytes(nbmax, topk, rp.sums);
        rp.err = err.as<int>();
        if ((e = launch_reduce(rp, nf, stream)) != cudaSuccess) {
            fail_all(std::string("reduce launch: ") + cudaGetErrorString(e));
            return false;
        }
        cudaMemcpyAsync(B.h_peaks.p, dpeaks.p, sizeof(DevPeak) * (size_t)nf * topk, cudaMemcpyDeviceToHost, stream);
    }
    if (enq) {
        cudaMemcpyAsync(B.h_err.p, err.p, sizeof(int), cudaMemcpyDeviceToHost, stream);
        cudaEventRecord(ev_step[par], stream);
    }
    // ---- retire the previous step, then hand this one over as the step in flight
    if (!retire_inflight()) return false;
    if (enq) {
        inflight = true;
        fl_parity = par;
        fl_finishing = std::move(finishing);
        std::lock_guard<std::mutex> lk(mu);
        ++steps;
    } else if (!finishing.empty()) {
        fail_all("internal: finishing requests without a step");
        return false;
    }
    return true;
}

// Waits for the step in flight and retires the requests it finished.
bool Server::retire_inflight()
{
    if (!inflight) return true;
    NvtxRange r_retire("bls.server.retire");
    inflight = false;
    cudaError_t e;
    if ((e = cudaEventSynchronize(ev_step[fl_parity])) != cudaSuccess) {
        fail_all(std::string("serving step: ") + cudaGetErrorString(e));
        return false;
    }
    StepBufs& B = sb[fl_parity];
    const int topk = P->d.topk;
    const int errw = *B.h_err.as<int>();
    std::lock_guard<std::mutex> lk(mu);
    const DevPeak* pk = B.h_peaks.as<DevPeak>();
    for (size_t q = 0; q < fl_finishing.size(); ++q) {
        Request* r = fl_finishing[q];
        r->finishing = false;
        if (r->cancel) {
            r->state = RState::Cancelled;
            r->status = BLS_ERR_CANCELLED;
            ++cancelled;
        } else if (errw) {
            r->state = RState::Failed;
            r->status = (errw & kErrInput) ? BLS_ERR_INVALID : BLS_ERR_INTERNAL;
            r->error = "device check failed";
            ++failed;
        } else {
            r->peaks.resize(topk);
            for (int e2 = 0; e2 < topk; ++e2) to_peak(pk[q * topk + e2], &r->peaks[e2]);
            r->state = RState::Done;
            r->status = BLS_OK;
            ++completed;
        }
        r->t_done = now_ms();
        latencies.push_back(r->t_done - r->t_submit);
        slots[r->slot] = nullptr;
        in_use -= r->bytes;
        cudaFreeAsync(r->dmem, stream);
        r->dmem = nullptr;
        r->t.clear(); r->t.shrink_to_fit();
        r->y.clear(); r->y.shrink_to_fit();
        r->dy.clear(); r->dy.shrink_to_fit();
        r->freqs.clear(); r->freqs.shrink_to_fit();
    }
    fl_finishing.clear();
    cv_done.notify_all();
    return true;
}

static bls_status server_start(bls_plan_impl* P, Server** out)
{
    std::lock_guard<std::mutex> lk(P->server_mu);
    if (P->server) { *out = P->server; return BLS_OK; }
    Server* S = new (std::nothrow) Server();
    if (!S) return set_error(BLS_ERR_NOMEM, "server allocation");
    S->P = P;
    S->max_active = P->d.max_active_requests > 0 ? P->d.max_active_requests : 64;
    if (P->d.step_point_freqs > 0) S->step_units = (double)P->d.step_point_freqs;
    if (const char* f = getenv("BLS_SERVER_FAIL_ALLOC_EVERY")) S->fail_every = atol(f);
    S->slots.assign(S->max_active, nullptr);
    cudaError_t e;
    const int topk = P->d.topk;
    const int M = S->max_active;
    if ((e = cudaSetDevice(P->device)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = S->cdesc.ensure(sizeof(CurveDesc) * M)) != cudaSuccess ||
        (e = S->ranges.ensure(sizeof(TileRange) * M)) != cudaSuccess ||
        (e = S->prefix.ensure(sizeof(long long) * 2 * M)) != cudaSuccess ||
        (e = S->counter.ensure(sizeof(int) * M + 64)) != cudaSuccess ||
        (e = S->err.ensure(64)) != cudaSuccess ||
        (e = S->dslots.ensure(sizeof(int) * 2 * M)) != cudaSuccess ||
        (e = S->dpeaks.ensure(sizeof(DevPeak) * (size_t)M * topk)) != cudaSuccess ||
        (e = S->h_cdesc.ensure(sizeof(CurveDesc) * M)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&S->ev_copy, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&S->ev_fork, cudaEventDisableTiming)) != cudaSuccess) {
        delete S;
        return cuda_fail(e, "server start");
    }
    for (int b = 0; b < 2; ++b) {
        Server::StepBufs& B = S->sb[b];
        if ((e = B.h_ranges.ensure(sizeof(TileRange) * M)) != cudaSuccess ||
            (e = B.h_prefix.ensure(sizeof(long long) * 2 * M)) != cudaSuccess ||
            (e = B.h_slots.ensure(sizeof(int) * 2 * M)) != cudaSuccess ||
            (e = B.h_peaks.ensure(sizeof(DevPeak) * (size_t)M * topk)) != cudaSuccess ||
            (e = B.h_err.ensure(64)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&S->ev_step[b], cudaEventDisableTiming)) != cudaSuccess) {
            delete S;
            return cuda_fail(e, "server start");
        }
    }
    for (int q = 0; q < Server::kClassStreams; ++q) {
        if ((e = cudaStreamCreateWithFlags(&S->cls_stream[q], cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&S->ev_join[q], cudaEventDisableTiming)) != cudaSuccess) {
            delete S;
            return cuda_fail(e, "server start");
        }
    }
    S->th = std::thread([S] { S->run(); });
    P->server = S;
    *out = S;
    return BLS_OK;
}

void server_destroy(bls_plan_impl* P)
{
    Server* S;
    {
        std::lock_guard<std::mutex> lk(P->server_mu);
        S = P->server;
        P->server = nullptr;
    }
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaSetDevice(P->device);
    if (S->stream) cudaStreamSynchronize(S->stream);
    if (S->copy_stream) cudaStreamSynchronize(S->copy_stream);
    for (Request* r : S->slots)
        if (r && r->dmem) cudaFreeAsync(r->dmem, S->stream);
    if (S->stream) cudaStreamSynchronize(S->stream);
    for (auto& kv : S->all) delete kv.second;
    DevBuf* bufs[] = {&S->cdesc, &S->ranges, &S->prefix, &S->counter, &S->err, &S->dslots, &S->dpeaks};
    for (DevBuf* b : bufs) b->release();
    S->h_cdesc.release();
    for (int b = 0; b < 2; ++b) {
        Server::StepBufs& B = S->sb[b];
        HostBuf* hb[] = {&B.h_ranges, &B.h_prefix, &B.h_slots, &B.h_peaks, &B.h_err};
        for (HostBuf* h : hb) h->release();
        if (S->ev_step[b]) cudaEventDestroy(S->ev_step[b]);
    }
    if (S->ev_copy) cudaEventDestroy(S->ev_copy);
    if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
    for (int q = 0; q < Server::kClassStreams; ++q) {
        if (S->cls_stream[q]) cudaStreamDestroy(S->cls_stream[q]);
        if (S->ev_join[q]) cudaEventDestroy(S->ev_join[q]);
    }
    if (S->ev_fork) cudaEventDestroy(S->ev_fork);
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
}

}  // namespace blsgpu

// ------------------------------------------------------------------------------ C ABI

extern "C" {

bls_status bls_submit(bls_plan* P, const bls_curve* c, uint64_t* ticket)
{
    if (!P || !c || !ticket) return set_error(BLS_ERR_INVALID, "NULL argument");
    const bool sequential = P->d.algo != BLS_ALGO_TILED;
    cudaError_t e = cudaSetDevice(P->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    CurveSpec s;
    bls_status st = resolve_curve(P, c, 0, &s);   // checks host values; device ones below
    if (st != BLS_OK) return st;
    Request* r = new (std::nothrow) Request();
    if (!r) return set_error(BLS_ERR_NOMEM, "request allocation");
    // copy the input (host or device) into the request
    r->t.resize(s.n);
    r->y.resize(s.n);
    if (s.dy) r->dy.resize(s.n);
    if (s.freqs) r->freqs.resize(s.nf);
    e = cudaMemcpy(r->t.data(), s.t, (size_t)s.n * 8, cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(r->y.data(), s.y, (size_t)s.n * 4, cudaMemcpyDefault);
    if (e == cudaSuccess && s.dy) e = cudaMemcpy(r->dy.data(), s.dy, (size_t)s.n * 4, cudaMemcpyDefault);
    if (e == cudaSuccess && s.freqs) e = cudaMemcpy(r->freqs.data(), s.freqs, (size_t)s.nf * 8, cudaMemcpyDefault);
    if (e != cudaSuccess) { delete r; return cuda_fail(e, "copying the request"); }
    if (s.t_dev || s.y_dev || s.dy_dev || s.f_dev) {   // device inputs: check the copied values
        for (int i = 0; i < s.n; ++i)
            if (!std::isfinite(r->t[i]) || !std::isfinite(r->y[i]) ||
                (s.dy && (!(r->dy[i] > 0.0f) || !std::isfinite(r->dy[i])))) {
                delete r;
                return set_error(BLS_ERR_INVALID, "point %d has a non-finite value or a non-positive error", i);
            }
        for (int j = 0; j < (int)r->freqs.size(); ++j)
            if (!(r->freqs[j] > 0.0) || !std::isfinite(r->freqs[j])) {
                delete r;
                return set_error(BLS_ERR_INVALID, "freqs[%d] is not a finite positive frequency", j);
            }
    }
    r->spec = s;
    r->spec.t = r->t.data();
    r->spec.y = r->y.data();
    r->spec.dy = s.dy ? r->dy.data() : nullptr;
    r->spec.freqs = s.freqs ? r->freqs.data() : nullptr;
    r->src = *c;
    r->src.t = r->t.data();
    r->src.y = r->y.data();
    r->src.dy = s.dy ? r->dy.data() : nullptr;
    r->src.freqs = s.freqs ? r->freqs.data() : nullptr;
    if (!sequential) {
        if ((st = fold_geometry(P, s.nb, s.kmin, s.kmax, &r->geom)) != BLS_OK) { delete r; return st; }
        const long long n2 = (s.n + 1) & ~1;
        r->bytes = up256((size_t)s.n * 8) + up256((size_t)s.n * 4) + (s.dy ? up256((size_t)s.n * 4) : 0) +
                   (s.freqs ? up256((size_t)s.nf * 8) : 0) + up256((size_t)(n2 + 2) * 16) +
                   up256((size_t)(n2 + 2) * 8) + up256((size_t)s.nf * 4);
        if (r->bytes > P->budget) {
            const size_t need = r->bytes;
            delete r;
            return set_error(BLS_ERR_NOMEM, "the request needs %zu device bytes, over the plan's budget", need);
        }
        r->ntiles = (s.nf + r->geom.T - 1) / r->geom.T;
        r->tile_cost = (double)r->geom.T * ((double)s.n + kEvalCost * (double)s.nb * (double)(s.kmax - s.kmin + 1));
    }
    Server* S = nullptr;
    if ((st = server_start(P, &S)) != BLS_OK) { delete r; return st; }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!S->fatal.empty()) { delete r; return set_error(BLS_ERR_CUDA, "server stopped: %s", S->fatal.c_str()); }
        r->id = S->next_id++;
        r->t_submit = now_ms();
        S->all[r->id] = r;
        S->queue.push_back(r);
        ++S->submitted;
        *ticket = r->id;
    }
    S->cv_work.notify_all();
    return BLS_OK;
}

bls_status bls_poll(bls_plan* P, uint64_t ticket, bls_peak* out, int timeout_ms)
{
    if (!P) return set_error(BLS_ERR_INVALID, "NULL plan");
    Server* S;
    {
        std::lock_guard<std::mutex> lk(P->server_mu);
        S = P->server;
    }
    if (!S) return set_error(BLS_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return set_error(BLS_ERR_INVALID, "unknown or retired ticket %llu", (unsigned long long)ticket);
    Request* r = it->second;
    auto finished = [&] { return r->state == RState::Done || r->state == RState::Failed || r->state == RState::Cancelled; };
    if (!finished()) {
        if (timeout_ms == 0) return BLS_PENDING;
        if (timeout_ms < 0) S->cv_done.wait(lk, finished);
        else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished))
            return set_error(BLS_ERR_TIMEOUT, "ticket %llu not finished after %d ms", (unsigned long long)ticket, timeout_ms);
    }
    bls_status st = r->status;
    if (r->state == RState::Done && out)
        for (size_t q = 0; q < r->peaks.size(); ++q) out[q] = r->peaks[q];
    if (r->state == RState::Failed) set_error(st, "%s", r->error.c_str());
    if (r->state == RState::Cancelled) { st = BLS_ERR_CANCELLED; set_error(st, "ticket was cancelled"); }
    S->all.erase(it);
    delete r;
    return st;
}

bls_status bls_cancel(bls_plan* P, uint64_t ticket)
{
    if (!P) return set_error(BLS_ERR_INVALID, "NULL plan");
    Server* S;
    {
        std::lock_guard<std::mutex> lk(P->server_mu);
        S = P->server;
    }
    if (!S) return set_error(BLS_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return set_error(BLS_ERR_INVALID, "unknown or retired ticket %llu", (unsigned long long)ticket);
    Request* r = it->second;
    if (r->state == RState::Queued) {          // still in the queue: cancelled at once
        S->queue.erase(std::remove(S->queue.begin(), S->queue.end(), r), S->queue.end());
        r->state = RState::Cancelled;
        r->status = BLS_ERR_CANCELLED;
        ++S->cancelled;
        S->cv_done.notify_all();
    } else if (r->state == RState::Active) {   // on the device: the scheduler retires it
        r->cancel = true;                      // at its next step
        S->cv_work.notify_all();
    }                                          // finished: nothing to cancel
    return BLS_OK;
}

bls_status bls_server_stats_get(bls_plan* P, bls_server_stats* out)
{
    if (!P || !out) return set_error(BLS_ERR_INVALID, "NULL argument");
    memset(out, 0, sizeof(*out));
    Server* S;
    {
        std::lock_guard<std::mutex> lk(P->server_mu);
        S = P->server;
    }
    if (!S) return BLS_OK;
    std::lock_guard<std::mutex> lk(S->mu);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->cancelled = S->cancelled;
    out->failed = S->failed;
    out->steps = S->steps;
    uint64_t act = 0;
    for (Request* r : S->slots) if (r) ++act;
    out->active = act;
    out->queued = S->queue.size();
    out->device_bytes_in_use = S->in_use;
    out->device_bytes_peak = S->peak_use;
    if (!S->latencies.empty()) {
        std::vector<double> v = S->latencies;
        auto pct = [&](double p) {
            size_t k = (size_t)std::min<double>((double)v.size() - 1, std::floor(p * (double)(v.size() - 1) + 0.5));
            std::nth_element(v.begin(), v.begin() + k, v.end());
            return v[k];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
    }
    return BLS_OK;
}

}  // extern "C"
