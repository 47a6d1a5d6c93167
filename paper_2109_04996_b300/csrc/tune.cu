// Autotuner of the fused apply's launch shape (elements per block, blocks per
// SM) for one operator, with a small JSON cache on disk.  The paper
// specializes its kernels by just-in-time compilation on the order (sections
// "Ecosystem" and "libCEED"); here the variants are compiled ahead of time and
// the tuner times them on the operator's own mesh with CUDA events.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "fem_internal.h"

namespace {

const int kBpsCandidates[] = {1, 2, 3, 4, 6, 0};  // 0 = occupancy maximum

int n_choices(const fem_op *) { return FEM_APPLY_CHOICES_MAX; }

std::string cache_key(const fem_op *op, int prec) {
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  int ebucket = 0;
  for (int64_t e = op->E; e > 1; e >>= 1) ebucket++;
  char buf[160];
  snprintf(buf, sizeof(buf), "sm_%d%d|P=%d|q=%d|kind=%d|colloc=%d|ncomp=%d|prec=%d|log2E=%d",
           major, minor, op->P, op->Q, op->kind, op->colloc ? 1 : 0, op->ncomp, prec, ebucket);
  return buf;
}

// Cache file: valid JSON with one entry per line,
//   {"fem_autotune_cache": 1, "entries": [
//   {"key": "...", "epb_choice": 0, "blocks_per_sm": 2, "us": 12.5},
//   ...
//   ]}
std::vector<std::string> read_entries(const char *path) {
  std::vector<std::string> out;
  FILE *f = fopen(path, "r");
  if (!f) return out;
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    std::string s(line);
    size_t a = s.find("{\"key\"");
    if (a == std::string::npos) continue;
    size_t b = s.rfind('}');
    if (b == std::string::npos || b < a) continue;
    out.push_back(s.substr(a, b - a + 1));
  }
  fclose(f);
  return out;
}

bool lookup(const std::vector<std::string> &entries, const std::string &key, int *choice,
            int *bps, double *us) {
  const std::string pat = "{\"key\": \"" + key + "\"";
  for (const std::string &e : entries) {
    if (e.compare(0, pat.size(), pat) != 0) continue;
    const char *c = strstr(e.c_str(), "\"epb_choice\":");
    const char *b = strstr(e.c_str(), "\"blocks_per_sm\":");
    const char *u = strstr(e.c_str(), "\"us\":");
    if (!c || !b || !u) continue;
    if (sscanf(c + 13, "%d", choice) != 1 || sscanf(b + 16, "%d", bps) != 1 ||
        sscanf(u + 5, "%lf", us) != 1)
      continue;
    return true;
  }
  return false;
}

int write_entries(const char *path, std::vector<std::string> entries, const std::string &key,
                  const std::string &entry) {
  const std::string pat = "{\"key\": \"" + key + "\"";
  bool replaced = false;
  for (std::string &e : entries)
    if (e.compare(0, pat.size(), pat) == 0) { e = entry; replaced = true; }
  if (!replaced) entries.push_back(entry);
  std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "w");
  if (!f) return FEM_EINVAL;
  fprintf(f, "{\"fem_autotune_cache\": 1, \"entries\": [\n");
  for (size_t i = 0; i < entries.size(); i++)
    fprintf(f, "%s%s\n", entries[i].c_str(), i + 1 < entries.size() ? "," : "");
  fprintf(f, "]}\n");
  fclose(f);
  if (rename(tmp.c_str(), path) != 0) return FEM_EINVAL;
  return FEM_OK;
}

int launch(fem_op *op, int prec, void *x, void *y, int choice, int bps) {
  if (prec == FEM_F64)
    return fem_launch_apply_f64_shape(op, (const double *)x, (double *)y, nullptr, op->E, nullptr,
                                      choice, bps);
  return fem_launch_apply_f32_shape(op, (const float *)x, (float *)y, nullptr, op->E, nullptr,
                                    choice, bps);
}

}  // namespace

extern "C" fem_status fem_op_set_launch_shape(fem_op *op, int prec, int epb_choice,
                                              int blocks_per_sm) {
  if (!op || (prec != FEM_F64 && prec != FEM_F32) || !fem_apply_choice_valid(op, prec, epb_choice) ||
      blocks_per_sm < 0) {
    fem_set_error("fem_op_set_launch_shape: invalid arguments");
    return FEM_EINVAL;
  }
  {
    const int rc = fem_ensure_choice_data(op, prec, epb_choice);
    if (rc) return rc;
  }
  op->tune_epb[prec] = epb_choice;
  op->tune_bps[prec] = blocks_per_sm;
  return FEM_OK;
}

extern "C" fem_status fem_op_autotune(fem_op *op, int prec, const char *cache_path,
                                      fem_tune_result *res) {
  if (!op || (prec != FEM_F64 && prec != FEM_F32)) {
    fem_set_error("fem_op_autotune: invalid arguments");
    return FEM_EINVAL;
  }
  if (prec == FEM_F32 && !op->d_qdata32) {
    fem_set_error("fem_op_autotune: operator was not created with FEM_F32");
    return FEM_EINVAL;
  }
  const std::string key = cache_key(op, prec);
  std::vector<std::string> entries;
  if (cache_path) {
    entries = read_entries(cache_path);
    int c, b;
    double us;
    if (lookup(entries, key, &c, &b, &us) && fem_apply_choice_valid(op, prec, c) && b >= 0) {
      {
        const int rc = fem_ensure_choice_data(op, prec, c);
        if (rc) return rc;
      }
      op->tune_epb[prec] = c;
      op->tune_bps[prec] = b;
      if (res) { res->epb_choice = c; res->blocks_per_sm = b; res->us = us; res->from_cache = 1; res->candidates = 0; }
      return FEM_OK;
    }
  }
  const size_t esz = prec == FEM_F64 ? 8 : 4;
  const size_t bytes = esz * (size_t)op->N * op->ncomp;
  void *x = nullptr, *y = nullptr;
  if (cudaMalloc(&x, bytes) != cudaSuccess || cudaMalloc(&y, bytes) != cudaSuccess) {
    cudaFree(x);
    cudaGetLastError();
    fem_set_error("fem_op_autotune: allocation of the timing vectors failed");
    return FEM_ENOMEM;
  }
  cudaStream_t s = op->stream();
  cudaEvent_t e0, e1;
  int rc = FEM_OK;
  FEM_CUDA_TRY(cudaEventCreate(&e0));
  FEM_CUDA_TRY(cudaEventCreate(&e1));
  cudaMemsetAsync(x, 0, bytes, s);
  double best = 1e300;
  int best_c = 0, best_b = 0, ncand = 0;
  for (int c = 0; c < n_choices(op) && rc == FEM_OK; c++) {
    if (!fem_apply_choice_valid(op, prec, c)) continue;
    if ((rc = fem_ensure_choice_data(op, prec, c))) break;
    for (int bps : kBpsCandidates) {
      // warm-up (also sets the kernel attributes)
      for (int w = 0; w < 2 && rc == FEM_OK; w++) rc = launch(op, prec, x, y, c, bps);
      if (rc == FEM_EINVAL) { rc = FEM_OK; cudaGetLastError(); break; }  // shape not valid here
      if (rc) break;
      const int reps = 5;
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps && rc == FEM_OK; r++) rc = launch(op, prec, x, y, c, bps);
      cudaEventRecord(e1, s);
      if (rc) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = FEM_ECUDA; break; }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double us = 1e3 * ms / reps;
      ncand++;
      if (us < best) { best = us; best_c = c; best_b = bps; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  if (rc) {
    if (rc == FEM_ECUDA) fem_set_error("fem_op_autotune: timing failed: %s", cudaGetErrorString(cudaGetLastError()));
    return rc;
  }
  op->tune_epb[prec] = best_c;
  op->tune_bps[prec] = best_b;
  if (res) { res->epb_choice = best_c; res->blocks_per_sm = best_b; res->us = best; res->from_cache = 0; res->candidates = ncand; }
  if (cache_path) {
    char buf[512];
    snprintf(buf, sizeof(buf), "{\"key\": \"%s\", \"epb_choice\": %d, \"blocks_per_sm\": %d, \"us\": %.3f}",
             key.c_str(), best_c, best_b, best);
    if (write_entries(cache_path, entries, key, buf) != FEM_OK) {
      fem_set_error("fem_op_autotune: could not write the cache file %s", cache_path);
      return FEM_EINVAL;
    }
  }
  return FEM_OK;
}
