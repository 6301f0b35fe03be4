// scheduler.h -- continuous-batching admission for the proof server (host).
//
// Block-proof jobs arrive every slot time (400 ms blocks, Section 3.1 and
// Figure "Proof pipelining across consecutive slots") and their proofs must
// land within the finality budget (Section 3.4; Definition "Two-Phase Proof
// Timeout" in Section 6 bounds how long a proof may be outstanding).  The
// scheduler keeps a FIFO of waiting jobs and starts the oldest one whenever a
// proving slot is idle and the device memory the job needs fits the budget;
// running jobs overlap on the device.  A job that waits longer than its
// deadline is dropped with a timeout.  Everything here is host logic over an
// abstract executor and clock, so it can be exercised without a GPU.
#pragma once
#include <stdint.h>

#include <deque>
#include <vector>

namespace ace {

struct SchedJob {
    uint64_t id = 0;
    double arrival = 0;     // seconds on the scheduler clock
    double deadline = 0;    // latest start time (arrival + max queue wait); <= 0: none
    size_t mem = 0;         // device bytes the job needs while it runs
    int slot = -1;
    int prio = 0;           // jobs already running when this one started
    double start = -1, finish = -1;
    int status = 0;         // 0 pending/ok, 1 unsat, -6 timeout, other < 0 error
    bool done = false;
};

// Executor: start(job, slot) -> 0 or error; poll(job) -> true when finished
// (and sets job.status).  Clock: now() in seconds.
template <class Executor, class Clock>
class Scheduler {
   public:
    Scheduler(Executor& ex, Clock& clock, int slots, size_t mem_budget)
        : ex_(ex), clock_(clock), busy_(slots, nullptr), budget_(mem_budget) {}

    // enqueue (the job keeps its arrival time)
    void submit(SchedJob* j) { queue_.push_back(j); }

    // one scheduling pass: retire finished jobs, time out expired waiters,
    // start waiting jobs on idle slots while memory allows.  Returns the
    // number of jobs that changed state.
    int step() {
        int changed = 0;
        double now = clock_.now();
        for (size_t s = 0; s < busy_.size(); s++) {
            SchedJob* j = busy_[s];
            if (j && ex_.poll(*j)) {
                j->finish = clock_.now();
                j->done = true;
                used_ -= j->mem;
                busy_[s] = nullptr;
                changed++;
            }
        }
        // FIFO: drop expired heads, then admit in order while possible
        while (!queue_.empty()) {
            SchedJob* j = queue_.front();
            if (j->deadline > 0 && now > j->deadline) {
                j->status = -6;
                j->done = true;
                j->finish = now;
                queue_.pop_front();
                changed++;
                continue;
            }
            int slot = idle_slot();
            if (slot < 0) break;
            if (j->mem > budget_) {  // can never fit
                j->status = -2;
                j->done = true;
                j->finish = now;
                queue_.pop_front();
                changed++;
                continue;
            }
            if (used_ + j->mem > budget_) break;  // wait for memory
            j->slot = slot;
            j->prio = 0;
            for (auto* b : busy_) j->prio += b != nullptr;
            j->start = clock_.now();
            int rc = ex_.start(*j, slot);
            queue_.pop_front();
            changed++;
            if (rc != 0) {
                j->status = rc;
                j->done = true;
                j->finish = j->start;
                continue;
            }
            used_ += j->mem;
            busy_[slot] = j;
            if (peak_used_ < used_) peak_used_ = used_;
            int running = 0;
            for (auto* b : busy_) running += b != nullptr;
            if (peak_running_ < running) peak_running_ = running;
        }
        return changed;
    }

    bool idle() const {
        if (!queue_.empty()) return false;
        for (auto* b : busy_)
            if (b) return false;
        return true;
    }
    size_t used() const { return used_; }
    size_t peak_used() const { return peak_used_; }
    int peak_running() const { return peak_running_; }
    size_t waiting() const { return queue_.size(); }

   private:
    int idle_slot() const {
        for (size_t s = 0; s < busy_.size(); s++)
            if (!busy_[s]) return (int)s;
        return -1;
    }
    Executor& ex_;
    Clock& clock_;
    std::deque<SchedJob*> queue_;
    std::vector<SchedJob*> busy_;
    size_t budget_;
    size_t used_ = 0, peak_used_ = 0;
    int peak_running_ = 0;
};

}  // namespace ace
