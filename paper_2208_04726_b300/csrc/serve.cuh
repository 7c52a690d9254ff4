// Serving runtime: many concurrent VO sessions with device-resident state,
// requests batched continuously into the solve launches.
//
// A session holds one problem in device memory owned by the library, admitted
// against the handle's memory budget: either a fixed graph (anchor, kk, jj)
// with its state (poses, patches) and factor buffers (target, weight), or a
// sliding window (Sec. 3.3, dpvo_ba_window) that grows by one frame per
// request and drops its oldest frame when full.  A request carries new
// factors for a fixed-graph session, or a new frame (patch centres) and the
// revisions and weights of the window's edges after the append.  The scheduler
// thread packs every pending request whose session is idle into one batch on
// one of its in-flight slots (a stream with its own workspace): the windows'
// appends (one batched call), one gather launch that reads every request's
// factors in place from page-locked host memory, the batched solve, and one
// launch that writes every status to page-locked memory.  Requests that
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
    dpvo_ba_problem dev{};        // device arrays (library-owned); a window session's come from its window
    char *mem = nullptr;          // one device allocation for all arrays (fixed-graph sessions)
    dpvo_ba_window *win = nullptr;  // the sliding window (window sessions)
    dpvo_ba_window_params wprm{};
    size_t bytes = 0;
    size_t max_edges = 0;         // edges the staging holds
    float *pinned_tw = nullptr;   // page-locked staging: target (or revision) then weight of the pending request
    float *pinned_xy = nullptr;   // window sessions: the new frame's patch centres
    int32_t *pinned_status = nullptr;
    bool busy = false;            // a request is queued or running
};

// One request's device work in a batch: its factors, read in place from
// page-locked host memory, and its status, written back to it.
struct GatherJob {
    const float2 *src_t, *src_w;  // host (page-locked): targets or revisions, weights
    float2 *dst_t, *dst_w;        // device: the session's (or window's) factor arrays
    int32_t n_edges;
    int32_t mode;                 // 0 replace target and weight, 1 target += revision and set weight, 2 none
    const int32_t *status_dev;
    int32_t *status_host;
};

struct Ticket {
    int64_t session = 0;
    int kind = 0;                 // 0 new factors, 1 new frame
    int n_new = 0;                // frame requests: patches of the new frame
    const float *src_t = nullptr, *src_w = nullptr, *src_xy = nullptr;   // page-locked sources
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
    dpvo_ba_dims max_dims{};                           // bound of every session's sizes
};

struct Slot {
    Server *srv = nullptr;
    dpvo_ba_handle *h = nullptr;  // private handle: workspace and descriptor staging
    cudaStream_t stream = nullptr;
    bool busy = false;
    std::vector<uint64_t> batch;  // tickets in flight on this slot
    GatherJob *jobs = nullptr;    // page-locked, max_batch entries, read by the gather and status launches
};

}  // namespace dpvo_serve
