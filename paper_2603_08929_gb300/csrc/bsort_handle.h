// Definition of the opaque bsort_handle (host state of one handle), shared by
// the translation units that create handles.
#pragma once

#include <cstdint>
#include <mutex>

#include "bsort_launch.h"

struct bsort_handle {
    using Ctl = bsort::Ctl;
    using Recorder = bsort::Recorder;
    int device = -1;
    // cached device buffers of the per-device default handles
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *stage = nullptr;  // device copy of host keys (bsort_keys_host)
    size_t stage_bytes = 0;
    // state of the last call
    Ctl *last_ctl = nullptr;
    cudaStream_t last_stream = nullptr;
    int last_path = 0;  // 0 none, 1 counting, 2 msd, 3 key-value msd
    bool last_inplace = false;
    size_t last_fixed_aux = 0;  // bytes of the last call's workspace outside the in-place buffers
    int last_key_bytes = 0;
    uint64_t last_n = 0;
    bsort::Tuning tune[2];  // MSD tuning for 4-byte [0] and 8-byte [1] keys (bsort_keys_ws)
    int stop_levels = 0;    // > 0: run only this many MSD levels (bsort_keys_partial_ws)
    bool profiling = false;
    bool events = false;
    Ctl *prof_ctl = nullptr;  // device slots: work counters of each recorded call
    int prof_path[BSORT_PROFILE_MAX_CALLS] = {0};
    int prof_key_bytes[BSORT_PROFILE_MAX_CALLS] = {0};
    uint64_t prof_n[BSORT_PROFILE_MAX_CALLS] = {0};
    // key-value calls: bytes of the value carried through the levels, and of
    // the value written per output element by the finish and fills (0: keys only)
    int prof_val_bytes[BSORT_PROFILE_MAX_CALLS] = {0};
    int prof_out_bytes[BSORT_PROFILE_MAX_CALLS] = {0};
    Recorder rec;
    std::mutex mu;
};
