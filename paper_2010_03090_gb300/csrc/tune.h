// Launch-configuration cache and autotuner (host side).
#pragma once
#include "internal.h"

namespace utf8gpu {

// Cached configuration for a GPU (name, SM count), defaults otherwise; the
// environment variables UTF8GPU_ROWS, UTF8GPU_BLOCKS_PER_SM,
// UTF8GPU_BATCH_ROWS and UTF8GPU_BATCH_BLOCKS_PER_SM override single fields,
// and UTF8GPU_TUNE_CACHE names a cache file read on first use.
LaunchCfg tuned_config(const char* gpu_name, int sm_count);

// Caps CTAs per SM at what the kernels' register and thread use allows.
void clamp_to_occupancy(LaunchCfg& cfg);

int run_autotune(int flags);
int tune_cache_load(const char* path);
int tune_cache_save(const char* path);

// current device helpers (api.cu)
LaunchCfg current_config();
void set_current_config(const LaunchCfg& cfg);
int current_sm_count();

// occupancy of the kernel instances (validate.cu, batch.cu)
int validate_blocks_per_sm(int rows);
int batch_blocks_per_sm(int rows);

}  // namespace utf8gpu
