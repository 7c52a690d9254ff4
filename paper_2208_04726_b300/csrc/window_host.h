// Host-side facts about a sliding window (window.cu) that the serving runtime
// needs: its device footprint for admission, its edge capacity for staging,
// and its edge count after an append, from the host mirror of its frame
// counts (no device access).  Internal to this library, not part of the C ABI.
#pragma once

#include <cstddef>

#include "dpvo_ba.h"

namespace dpvo_win_host {

// Bytes of device memory dpvo_ba_window_create allocates for these parameters.
size_t device_bytes(const dpvo_ba_window_params &p);
// Edges the window can hold at most.
size_t max_edges(const dpvo_ba_window_params &p);
// Edges the window holds after appending a frame of n_new patches.
int edges_after(const dpvo_ba_window *w, int n_new);
// Frames and patches the window holds now.
void sizes(const dpvo_ba_window *w, int *n_frames, int *n_patches, int *n_edges);

}  // namespace dpvo_win_host
