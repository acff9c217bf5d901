// Launch-configuration autotuner and its cache.
//
// The tunables are the tile height (rows of 512 bytes per warp tile), the
// number of resident CTAs per SM of the persistent grid, and the same two for
// the batch kernel.  run_autotune times every candidate with CUDA events on
// synthetic text generated on the device (a mix of ASCII, 2-, 3- and 4-byte
// characters, and a batch of uneven strings over it) and keeps the fastest.
// Results are cached per (GPU name, SM count) and can be saved to / loaded
// from a small JSON file.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>

#include "internal.h"
#include "tune.h"
#include "utf8gpu.h"

namespace utf8gpu {

namespace {

std::mutex g_mu;
std::map<std::string, LaunchCfg> g_cache;  // key: "<gpu name>|<sm count>"

std::string key_of(const char* name, int sms) { return std::string(name) + "|" + std::to_string(sms); }

int env_int(const char* name, int fallback) {
  const char* v = getenv(name);
  if (!v || !*v) return fallback;
  return atoi(v);
}

void apply_env(LaunchCfg& c) {
  c.rows = env_int("UTF8GPU_ROWS", c.rows);
  c.blocks_per_sm = env_int("UTF8GPU_BLOCKS_PER_SM", c.blocks_per_sm);
  c.batch_rows = env_int("UTF8GPU_BATCH_ROWS", c.batch_rows);
  c.batch_blocks_per_sm = env_int("UTF8GPU_BATCH_BLOCKS_PER_SM", c.batch_blocks_per_sm);
}

}  // namespace

// Each 16-byte granule holds whole characters: 16 ASCII, 8 two-byte, 5
// three-byte + 1 ASCII, or 4 four-byte characters, picked by a hash.
__global__ void synth_text_kernel(uint8_t* out, uint64_t granules, uint32_t seed) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= granules) return;
  uint32_t h = (uint32_t)g * 0x9E3779B9u ^ seed;
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12;
  uint8_t b[16];
  switch (h & 3) {
    case 0:
      for (int i = 0; i < 16; ++i) b[i] = (uint8_t)(0x61 + ((h >> (i & 7)) & 15));
      break;
    case 1:
      for (int i = 0; i < 8; ++i) { b[2 * i] = 0xC3; b[2 * i + 1] = (uint8_t)(0x80 + ((h >> i) & 63)); }
      break;
    case 2:
      for (int i = 0; i < 5; ++i) {
        b[3 * i] = 0xE4 + (i & 1); b[3 * i + 1] = (uint8_t)(0x80 + ((h >> i) & 63));
        b[3 * i + 2] = (uint8_t)(0x80 + ((h >> (i + 3)) & 63));
      }
      b[15] = 0x20;
      break;
    default:
      for (int i = 0; i < 4; ++i) {
        b[4 * i] = 0xF0; b[4 * i + 1] = 0x9F; b[4 * i + 2] = (uint8_t)(0x80 + ((h >> i) & 63));
        b[4 * i + 3] = (uint8_t)(0x80 + ((h >> (i + 5)) & 63));
      }
  }
  uint4 v;
  memcpy(&v, b, 16);
  reinterpret_cast<uint4*>(out)[g] = v;
}

// String ends at granule boundaries (every string is whole characters):
// lengths 16 * (1 .. 64) granules, hashed.
__global__ void synth_offsets_kernel(int64_t* offsets, int64_t count, uint64_t total_granules) {
  // single-thread prefix: tuning batches are small enough
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t pos = 0;
  offsets[0] = 0;
  for (int64_t i = 0; i < count; ++i) {
    uint32_t h = (uint32_t)i * 0x9E3779B9u;
    h ^= h >> 13; h *= 0x5BD1E995u; h ^= h >> 15;
    int64_t len = 16 * (1 + (int64_t)(h % 64));
    if ((uint64_t)(pos + len) > total_granules * 16) len = 0;
    pos += len;
    offsets[i + 1] = pos;
  }
}

LaunchCfg tuned_config(const char* gpu_name, int sm_count) {
  static std::once_flag env_cache;
  std::call_once(env_cache, [] {
    const char* path = getenv("UTF8GPU_TUNE_CACHE");
    if (path && *path) tune_cache_load(path);
  });
  std::lock_guard<std::mutex> lock(g_mu);
  LaunchCfg c;
  auto it = g_cache.find(key_of(gpu_name, sm_count));
  if (it != g_cache.end()) c = it->second;
  apply_env(c);
  return c;
}

// The staged 8-row passes run where this device's kernels accept their shared
// memory and the grid's CTAs per SM fit beside it; else the register form.
// UTF8GPU_STAGED=0 keeps the register form.
static void apply_staged(LaunchCfg& cfg) {
  cfg.staged = cfg.rows == 8 && env_int("UTF8GPU_STAGED", 1) != 0 &&
               prepare_staged_kernels() == cudaSuccess &&
               prepare_chunk_staged() == cudaSuccess &&
               cfg.blocks_per_sm <= staged_blocks_per_sm();
}

void clamp_to_occupancy(LaunchCfg& cfg) {
  if (cfg.rows != 2 && cfg.rows != 4 && cfg.rows != 8) cfg.rows = 8;
  if (cfg.batch_rows != 2 && cfg.batch_rows != 4 && cfg.batch_rows != 8) cfg.batch_rows = 8;
  const int v = validate_blocks_per_sm(cfg.rows);
  int b = batch_blocks_per_sm(cfg.batch_rows);
  if (b < 1 && cfg.batch_rows != 2) {  // no room for the larger rings
    cfg.batch_rows = 2;
    b = batch_blocks_per_sm(2);
  }
  if (b < 1) b = 1;
  if (cfg.blocks_per_sm < 1 || cfg.blocks_per_sm > v) cfg.blocks_per_sm = v;
  if (cfg.batch_blocks_per_sm < 1 || cfg.batch_blocks_per_sm > b) cfg.batch_blocks_per_sm = b;
  apply_staged(cfg);
}

static float time_ms(cudaStream_t st, cudaEvent_t a, cudaEvent_t b, int reps,
                     const LaunchCfg& cfg, int sms, bool batch, const uint8_t* data,
                     uint64_t bytes, const int64_t* offsets, int64_t count, uint8_t* out) {
  for (int i = 0; i < 3; ++i) {
    if (batch) launch_batch(data, offsets, count, out, cfg, sms, st);
    else launch_validate(data, bytes, out, cfg, sms, st);
  }
  cudaEventRecord(a, st);
  for (int i = 0; i < reps; ++i) {
    if (batch) launch_batch(data, offsets, count, out, cfg, sms, st);
    else launch_validate(data, bytes, out, cfg, sms, st);
  }
  cudaEventRecord(b, st);
  cudaEventSynchronize(b);
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  return ms / reps;
}

int run_autotune(int flags) {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return UTF8_ERR_CUDA;
  const std::string key = key_of(prop.name, prop.multiProcessorCount);
  if (!(flags & 1)) {
    bool cached = false;
    LaunchCfg c;
    {
      std::lock_guard<std::mutex> lock(g_mu);
      auto it = g_cache.find(key);
      if (it != g_cache.end()) { cached = true; c = it->second; }
    }
    if (cached) {
      set_current_config(c);
      return UTF8_OK;
    }
  }
  const int sms = prop.multiProcessorCount;
  const uint64_t bytes = 512ull << 20;  // larger than L2
  const uint64_t granules = bytes / 16;
  const int64_t count = 200000;
  uint8_t* data = nullptr;
  int64_t* offsets = nullptr;
  uint8_t* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaMalloc(&data, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&offsets, (count + 1) * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&out, count);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  LaunchCfg best = current_config();
  if (e == cudaSuccess) {
    synth_text_kernel<<<(unsigned)((granules + 255) / 256), 256, 0, st>>>(data, granules, 20100309u);
    synth_offsets_kernel<<<1, 1, 0, st>>>(offsets, count, granules);
    e = cudaStreamSynchronize(st);
  }
  if (e == cudaSuccess) {
    float best_single = 1e30f, best_batch = 1e30f;
    const int rows_c[3] = {2, 4, 8};
    const int brows_c[3] = {2, 4, 8};
    const int bps_c[4] = {2, 4, 6, 8};
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 4; ++k) {
        LaunchCfg c = best;
        c.rows = rows_c[r];
        c.blocks_per_sm = bps_c[k];
        if (c.blocks_per_sm > validate_blocks_per_sm(c.rows)) continue;
        apply_staged(c);
        const float ms = time_ms(st, a, b, 10, c, sms, false, data, bytes, offsets, count, out);
        if (ms < best_single) { best_single = ms; best.rows = c.rows; best.blocks_per_sm = c.blocks_per_sm; }
      }
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 4; ++k) {
        LaunchCfg c = best;
        c.batch_rows = brows_c[r];
        c.batch_blocks_per_sm = bps_c[k];
        if (c.batch_blocks_per_sm > batch_blocks_per_sm(c.batch_rows)) continue;
        const float ms = time_ms(st, a, b, 10, c, sms, true, data, bytes, offsets, count, out);
        if (ms < best_batch) { best_batch = ms; best.batch_rows = c.batch_rows; best.batch_blocks_per_sm = c.batch_blocks_per_sm; }
      }
    e = cudaGetLastError();
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) cudaStreamDestroy(st);
  cudaFree(data);
  cudaFree(offsets);
  cudaFree(out);
  if (e != cudaSuccess) return UTF8_ERR_CUDA;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[key] = best;
  }
  set_current_config(best);
  return UTF8_OK;
}

int tune_cache_save(const char* path) {
  std::lock_guard<std::mutex> lock(g_mu);
  FILE* f = fopen(path, "w");
  if (!f) return UTF8_ERR_INVALID_ARG;
  fprintf(f, "{\"entries\": [\n");
  size_t i = 0;
  for (const auto& kv : g_cache) {
    const size_t bar = kv.first.rfind('|');
    fprintf(f,
            "  {\"gpu\": \"%s\", \"sms\": %s, \"rows\": %d, \"blocks_per_sm\": %d, "
            "\"batch_rows\": %d, \"batch_blocks_per_sm\": %d}%s\n",
            kv.first.substr(0, bar).c_str(), kv.first.substr(bar + 1).c_str(), kv.second.rows,
            kv.second.blocks_per_sm, kv.second.batch_rows, kv.second.batch_blocks_per_sm,
            ++i < g_cache.size() ? "," : "");
  }
  fprintf(f, "]}\n");
  fclose(f);
  return UTF8_OK;
}

// Reads the entries written by tune_cache_save (one object per line).
int tune_cache_load(const char* path) {
  FILE* f = fopen(path, "r");
  if (!f) return UTF8_ERR_INVALID_ARG;
  char line[1024];
  std::map<std::string, LaunchCfg> got;
  while (fgets(line, sizeof line, f)) {
    const char* g = strstr(line, "\"gpu\": \"");
    if (!g) continue;
    g += 8;
    const char* ge = strchr(g, '"');
    if (!ge) continue;
    const std::string name(g, ge - g);
    int sms = 0;
    LaunchCfg c;
    if (sscanf(ge + 1,
               ", \"sms\": %d, \"rows\": %d, \"blocks_per_sm\": %d, \"batch_rows\": %d, "
               "\"batch_blocks_per_sm\": %d",
               &sms, &c.rows, &c.blocks_per_sm, &c.batch_rows, &c.batch_blocks_per_sm) == 5)
      got[key_of(name.c_str(), sms)] = c;
  }
  fclose(f);
  std::lock_guard<std::mutex> lock(g_mu);
  for (const auto& kv : got) g_cache[kv.first] = kv.second;
  return UTF8_OK;
}

}  // namespace utf8gpu
