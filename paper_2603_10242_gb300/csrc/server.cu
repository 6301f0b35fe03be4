// server.cu -- the proof server: block-proof jobs are proved as they arrive
// (the builder's Phase 2 loop, Section 3.3 Algorithm 3 GPUProofPipeline:
// wait for a published block, prove it, publish the certificate), with
// continuous batching.  Jobs that arrive while others are on the GPU start as
// soon as a proving slot is idle and the device memory they need fits the
// budget; their work overlaps on the device.  One host thread owns the
// context while the server runs; callers submit and poll from any thread.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "pk.h"
#include "scheduler.h"


using namespace ace;

namespace {

struct ServerJob : SchedJob {
    const ace_pk* pk = nullptr;
    const ace_fr* z = nullptr;  // host witness, valid until the job is done
    fr_t r, s;
    uint8_t proof[256];
    double wall_arrival = 0;
};

struct SlotIo {
    fr_t* d_z = nullptr;
    size_t z_cap = 0;
    uint32_t* d_proof = nullptr;
    int32_t* d_status = nullptr;
    uint8_t* h_proof = nullptr;   // pinned
    int32_t* h_status = nullptr;  // pinned
    cudaEvent_t done = nullptr;
};

struct SteadyClock {
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

struct CudaExecutor {
    ace_ctx* ctx = nullptr;
    std::vector<SlotIo>* io = nullptr;
    int start(SchedJob& sj, int slot) {
        ServerJob& j = static_cast<ServerJob&>(sj);
        SlotIo& s = (*io)[slot];
        ProveSlot& sl = ctx->slots[slot];
        // jobs admitted while others run get lower stream priorities, so the
        // device keeps serving jobs roughly in admission order
        int prio = j.prio < PRIO_LEVELS ? j.prio : PRIO_LEVELS - 1;
        cudaStream_t m = sl.lv[prio].main;
        size_t zb = (size_t)j.pk->m * sizeof(fr_t);
        if (zb > s.z_cap) return ACE_E_OOM;
        // the slot's previous job may still read d_z
        if (cudaStreamWaitEvent(m, sl.ev_done, 0) != cudaSuccess) return ACE_E_CUDA;
        if (cudaMemcpyAsync(s.d_z, j.z, zb, cudaMemcpyHostToDevice, m) != cudaSuccess) return ACE_E_CUDA;
        int rc = prove_run(ctx, slot, prio, j.pk, s.d_z, j.r, j.s, s.d_proof, s.d_status, m, false);
        if (rc != ACE_OK) return rc;
        if (cudaMemcpyAsync(s.h_proof, s.d_proof, 256, cudaMemcpyDeviceToHost, m) != cudaSuccess ||
            cudaMemcpyAsync(s.h_status, s.d_status, 4, cudaMemcpyDeviceToHost, m) != cudaSuccess ||
            cudaEventRecord(s.done, m) != cudaSuccess)
            return ACE_E_CUDA;
        return ACE_OK;
    }
    bool poll(SchedJob& sj) {
        ServerJob& j = static_cast<ServerJob&>(sj);
        SlotIo& s = (*io)[j.slot];
        cudaError_t e = cudaEventQuery(s.done);
        if (e == cudaErrorNotReady) return false;
        if (e != cudaSuccess) {
            j.status = ACE_E_CUDA;
            return true;
        }
        memcpy(j.proof, s.h_proof, 256);
        j.status = *s.h_status ? 1 : 0;
        return true;
    }
};

}  // namespace

struct ace_server {
    ace_ctx* ctx = nullptr;
    int slots = 0;
    size_t budget = 0;
    double max_wait = 0;
    std::vector<SlotIo> io;
    CudaExecutor ex;
    SteadyClock clk;
    Scheduler<CudaExecutor, SteadyClock>* sched = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::vector<ServerJob*> incoming;
    std::unordered_map<uint64_t, ServerJob*> jobs;
    uint64_t next_id = 1;
    uint64_t submitted = 0, finished = 0, timeouts = 0;
    bool stop = false;
    int thread_error = 0;
    std::thread th;

    // the scheduling loop: hand new jobs to the scheduler, run one pass
    // (retire, time out, admit) under the lock, sleep briefly when idle
    void loop() {
        cudaSetDevice(ctx->device);
        for (;;) {
            int changed = 0;
            {
                std::lock_guard<std::mutex> g(mu);
                if (stop && incoming.empty() && sched->idle()) return;
                for (auto* j : incoming) sched->submit(j);
                incoming.clear();
                changed = sched->step();
            }
            if (changed) cv.notify_all();
            else std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
    }
};

extern "C" {

int ace_server_create(ace_ctx* ctx, const ace_pk* max_pk, int slots, size_t hbm_budget_bytes, double max_queue_wait_s,
                      ace_server** out) {
    clear_error();
    if (!ctx || !max_pk || !out || slots < 1 || slots > MAX_SLOTS) {
        set_error("ace_server_create: bad argument (slots must be 1..%d)", MAX_SLOTS);
        return ACE_E_ARG;
    }
    *out = nullptr;
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    ace_server* sv = new ace_server();
    sv->ctx = ctx;
    ctx_ref(ctx);
    sv->slots = slots;
    sv->max_wait = max_queue_wait_s;
    sv->io.resize(slots);
    // slot scratch sized for the largest key up front, so nothing grows (and
    // synchronises the device) while jobs run
    size_t per_job = max_pk->m * sizeof(fr_t);
    for (int k = 0; k < PROVE_ARENAS; k++) per_job += prove_slot_bytes(max_pk, k);
    sv->budget = hbm_budget_bytes ? hbm_budget_bytes : per_job * slots;
    auto fail = [&](int rc) {
        for (auto& s : sv->io) {
            if (s.d_z) cudaFree(s.d_z);
            if (s.d_proof) cudaFree(s.d_proof);
            if (s.h_proof) cudaFreeHost(s.h_proof);
            if (s.h_status) cudaFreeHost(s.h_status);
            if (s.done) cudaEventDestroy(s.done);
        }
        delete sv;
        ctx_unref(ctx);
        return rc;
    };
    for (int q = 0; q < slots; q++) {
        int rc = slot_ready(ctx, q);
        for (int k = 0; k < PROVE_ARENAS && rc == ACE_OK; k++) rc = slot_arena_ensure(ctx, q, k, prove_slot_bytes(max_pk, k));
        if (rc != ACE_OK) return fail(rc);
        SlotIo& s = sv->io[q];
        s.z_cap = max_pk->m * sizeof(fr_t);
        if (cudaMalloc(&s.d_z, s.z_cap) != cudaSuccess || cudaMalloc(&s.d_proof, 512) != cudaSuccess ||
            cudaMallocHost(&s.h_proof, 256) != cudaSuccess || cudaMallocHost(&s.h_status, 16) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            set_error("ace_server_create: device or pinned allocation failed");
            return fail(ACE_E_OOM);
        }
        s.d_status = (int32_t*)((char*)s.d_proof + 256);
    }
    sv->ex.ctx = ctx;
    sv->ex.io = &sv->io;
    sv->sched = new Scheduler<CudaExecutor, SteadyClock>(sv->ex, sv->clk, slots, sv->budget);
    sv->th = std::thread([sv]() { sv->loop(); });
    *out = sv;
    return ACE_OK;
}

int ace_server_submit(ace_server* sv, const ace_pk* pk, const ace_fr* z_host, const ace_fr* r, const ace_fr* s,
                      uint64_t* job_id) {
    clear_error();
    if (!sv || !pk || !z_host || !r || !s || !job_id) {
        set_error("ace_server_submit: NULL argument");
        return ACE_E_ARG;
    }
    if ((size_t)pk->m * sizeof(fr_t) > sv->io[0].z_cap) {
        set_error("ace_server_submit: witness of %llu values exceeds the server's largest key",
                  (unsigned long long)pk->m);
        return ACE_E_ARG;
    }
    ServerJob* j = new ServerJob();
    j->pk = pk;
    j->z = z_host;
    memcpy(j->r.v, r->l, 32);
    memcpy(j->s.v, s->l, 32);
    if (fe_geq_mod(j->r) || fe_geq_mod(j->s)) {
        delete j;
        set_error("ace_server_submit: r and s must be canonical");
        return ACE_E_ARG;
    }
    size_t mem = pk->m * sizeof(fr_t);
    for (int k = 0; k < PROVE_ARENAS; k++) mem += prove_slot_bytes(pk, k);
    j->mem = mem;
    std::lock_guard<std::mutex> g(sv->mu);
    j->id = sv->next_id++;
    j->arrival = sv->clk.now();
    j->wall_arrival = j->arrival;
    j->deadline = sv->max_wait > 0 ? j->arrival + sv->max_wait : 0;
    sv->jobs[j->id] = j;
    sv->incoming.push_back(j);
    sv->submitted++;
    *job_id = j->id;
    return ACE_OK;
}

static int take_result(ace_server* sv, ServerJob* j, uint8_t* proof_out, double* latency_ms) {
    if (latency_ms) *latency_ms = (j->finish - j->arrival) * 1e3;
    int st = j->status;
    if (proof_out && st == 0) memcpy(proof_out, j->proof, 256);
    sv->jobs.erase(j->id);
    sv->finished++;
    if (st == -6) sv->timeouts++;
    delete j;
    if (st == 1) {
        set_error("job: witness does not satisfy the R1CS");
        return ACE_E_UNSAT;
    }
    if (st == -6) {
        set_error("job: waited longer than the queue deadline");
        return ACE_E_TIMEOUT;
    }
    if (st < 0) {
        set_error("job failed with code %d", st);
        return st;
    }
    return ACE_OK;
}

int ace_server_poll(ace_server* sv, uint64_t job_id, uint8_t proof_out[256], double* latency_ms) {
    clear_error();
    if (!sv) return ACE_E_ARG;
    std::lock_guard<std::mutex> g(sv->mu);
    auto it = sv->jobs.find(job_id);
    if (it == sv->jobs.end()) {
        set_error("ace_server_poll: unknown job %llu", (unsigned long long)job_id);
        return ACE_E_ARG;
    }
    if (!it->second->done) return ACE_E_BUSY;
    return take_result(sv, it->second, proof_out, latency_ms);
}

int ace_server_wait(ace_server* sv, uint64_t job_id, uint8_t proof_out[256], double* latency_ms, double timeout_s) {
    clear_error();
    if (!sv) return ACE_E_ARG;
    std::unique_lock<std::mutex> g(sv->mu);
    auto it = sv->jobs.find(job_id);
    if (it == sv->jobs.end()) {
        set_error("ace_server_wait: unknown job %llu", (unsigned long long)job_id);
        return ACE_E_ARG;
    }
    ServerJob* j = it->second;
    bool ok = sv->cv.wait_for(g, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9),
                              [&]() { return j->done; });
    if (!ok) return ACE_E_BUSY;
    return take_result(sv, j, proof_out, latency_ms);
}

// stats: submitted, finished (collected), timeouts, waiting, peak running
// jobs, peak device bytes admitted, budget, slots
int ace_server_stats(ace_server* sv, uint64_t out[8]) {
    if (!sv || !out) return ACE_E_ARG;
    std::lock_guard<std::mutex> g(sv->mu);
    out[0] = sv->submitted;
    out[1] = sv->finished;
    out[2] = sv->timeouts;
    out[3] = sv->sched->waiting() + sv->incoming.size();
    out[4] = (uint64_t)sv->sched->peak_running();
    out[5] = sv->sched->peak_used();
    out[6] = sv->budget;
    out[7] = (uint64_t)sv->slots;
    return ACE_OK;
}

int ace_server_destroy(ace_server* sv) {
    if (!sv) return ACE_OK;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stop = true;
    }
    if (sv->th.joinable()) sv->th.join();
    cudaSetDevice(sv->ctx->device);
    cudaDeviceSynchronize();
    for (auto& kv : sv->jobs) delete kv.second;
    for (auto& s : sv->io) {
        cudaFree(s.d_z);
        cudaFree(s.d_proof);
        cudaFreeHost(s.h_proof);
        cudaFreeHost(s.h_status);
        cudaEventDestroy(s.done);
    }
    delete sv->sched;
    ace_ctx* ctx = sv->ctx;
    delete sv;
    ctx_unref(ctx);
    return ACE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Scheduler simulation with a virtual clock (no GPU): the same admission code
// driven by jobs of given arrival, duration and memory.
// ---------------------------------------------------------------------------
namespace {
struct SimClock {
    double t = 0;
    double now() const { return t; }
};
struct SimExecutor {
    const double* duration = nullptr;
    SimClock* clock = nullptr;
    int start(SchedJob&, int) { return 0; }
    bool poll(SchedJob& j) { return clock->t >= j.start + duration[j.id]; }
};
}  // namespace

extern "C" int ace_debug_scheduler_sim(int slots, size_t budget, size_t n, const double* arrival,
                                       const double* duration, const size_t* mem, double max_wait, double* start_out,
                                       double* finish_out, int32_t* status_out, uint64_t* peaks, int32_t* prio_out) {
    if (slots < 1 || !arrival || !duration || !mem || !start_out || !finish_out || !status_out || !peaks)
        return ACE_E_ARG;
    SimClock clock;
    SimExecutor ex;
    ex.duration = duration;
    ex.clock = &clock;
    Scheduler<SimExecutor, SimClock> sched(ex, clock, slots, budget);
    std::vector<SchedJob> jobs(n);
    size_t next = 0;
    for (;;) {
        while (next < n && arrival[next] <= clock.t) {
            SchedJob& j = jobs[next];
            j.id = next;
            j.arrival = arrival[next];
            j.deadline = max_wait > 0 ? arrival[next] + max_wait : 0;
            j.mem = mem[next];
            sched.submit(&j);
            next++;
        }
        while (sched.step()) {
        }
        if (next >= n && sched.idle()) break;
        // advance to the next event: an arrival, a finish or a deadline
        double tn = 1e300;
        if (next < n) tn = arrival[next];
        for (auto& j : jobs) {
            if (j.start >= 0 && !j.done) tn = tn < j.start + duration[j.id] ? tn : j.start + duration[j.id];
            if (j.start < 0 && !j.done && j.deadline > 0 && j.arrival <= clock.t)
                tn = tn < j.deadline + 1e-9 ? tn : j.deadline + 1e-9;
        }
        if (tn >= 1e299) break;
        clock.t = tn > clock.t ? tn : clock.t;
    }
    for (size_t i = 0; i < n; i++) {
        start_out[i] = jobs[i].start;
        finish_out[i] = jobs[i].finish;
        status_out[i] = jobs[i].status;
        if (prio_out) prio_out[i] = jobs[i].prio;
    }
    peaks[0] = (uint64_t)sched.peak_running();
    peaks[1] = sched.peak_used();
    return ACE_OK;
}
