// Serving runtime: many concurrent VO sessions with device-resident state,
// requests batched continuously into the solve launches.
//
// A session holds one problem's graph (anchor, kk, jj), state (poses,
// patches) and factor buffers (target, weight) in device memory owned by the
// library, admitted against the handle's memory budget.  A request carries a
// new set of factors (host memory) for one session; the scheduler thread packs
// every pending request whose session is idle into one batched solve on one of
// its in-flight slots (a stream with its own workspace), so requests that
// arrive while a batch runs go into the next batch and consecutive batches
// overlap on the device.  Completion is timestamped by a host callback on the
// slot's stream.  Every wait is bounded.
#pragma once

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace dpvo_serve {

using Clock = std::chrono::steady_clock;

struct Session {
    int64_t id = 0;
    dpvo_ba_dims dims{};
    dpvo_ba_problem dev{};        // device arrays (library-owned)
    char *mem = nullptr;          // one device allocation for all arrays
    size_t bytes = 0;
    float *pinned_tw = nullptr;   // pinned staging: target then weight of the pending request
    int32_t *pinned_status = nullptr;
    bool busy = false;            // a request is queued or running
};

struct Ticket {
    int64_t session = 0;
    Clock::time_point submitted;
    Clock::time_point done_at;
    bool done = false;
    int32_t status = 0;
};

struct Slot;

struct Server {
    dpvo_ba_handle *owner = nullptr;
    int device = 0;
    int max_batch = 64;
    std::vector<Slot *> slots;
    std::thread thread;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    bool running = false;
    std::deque<uint64_t> pending;                      // ticket ids, FIFO
    std::unordered_map<uint64_t, Ticket> tickets;
    std::unordered_map<int64_t, Session *> sessions;
    uint64_t next_ticket = 1;
    int64_t next_session = 1;
    size_t used_bytes = 0;
    size_t budget = 0;
    int launch_error = 0;
};

struct Slot {
    Server *srv = nullptr;
    dpvo_ba_handle *h = nullptr;  // private handle: workspace and descriptor staging
    cudaStream_t stream = nullptr;
    bool busy = false;
    std::vector<uint64_t> batch;  // tickets in flight on this slot
};

}  // namespace dpvo_serve
