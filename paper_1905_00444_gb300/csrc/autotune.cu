// Autotuner for the contraction-step kernels: for every distinct step shape of a plan
// (N, K, NL, Sd) it times each compatible FP32 tile variant on the GPU (CUDA events, on the
// caller's workspace) and, for plans in a tensor-core precision, the tensor-core kernel as
// one more candidate; the fastest goes into a JSON cache keyed by the shape, the plan's
// precision and its tensor-core flags.  qfx_plan_create with qfx_plan_opts.autotune_cache
// applies the cached choices; shapes not in the cache keep the planner's default.  Format:
//   {"qfx_autotune": 1, "entries": [
//     {"N": 256, "K": 256, "NL": 256, "Sd": 1048576, "prec": 0, "tc_flags": 0,
//      "variant": 0, "ms": 1.23}, ...]}
// A variant of 10 or more stands for the tensor-core kernel of the entry's precision.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "qfx_internal.h"

namespace qfx {
namespace {

using Key = std::tuple<int64_t, int64_t, int64_t, int64_t, int, int>;   // N, K, NL, Sd, prec, tc flags
struct Entry {
  int variant;
  double ms;
};

bool number_after(const std::string& s, const std::string& key, double* v) {
  const std::string pat = "\"" + key + "\"";
  const size_t p = s.find(pat);
  if (p == std::string::npos) return false;
  size_t q = s.find(':', p + pat.size());
  if (q == std::string::npos) return false;
  try {
    *v = std::stod(s.substr(q + 1));
  } catch (...) {
    return false;
  }
  return true;
}

std::map<Key, Entry> read_cache(const char* path) {
  std::map<Key, Entry> out;
  if (!path) return out;
  std::ifstream f(path);
  if (!f) return out;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string text = ss.str();
  const size_t list = text.find("\"entries\"");
  if (list == std::string::npos) return out;
  size_t pos = list;
  for (;;) {
    const size_t a = text.find('{', pos);
    if (a == std::string::npos) break;
    const size_t b = text.find('}', a);
    if (b == std::string::npos) break;
    const std::string e = text.substr(a, b - a + 1);
    double N, K, NL, Sd, v, ms = 0, prec = 0, fl = 0;
    if (number_after(e, "N", &N) && number_after(e, "K", &K) && number_after(e, "NL", &NL) &&
        number_after(e, "Sd", &Sd) && number_after(e, "variant", &v)) {
      number_after(e, "ms", &ms);
      number_after(e, "prec", &prec);
      number_after(e, "tc_flags", &fl);
      if (v >= 0 && (v < 10 || (prec > 0 && v == kVariantTcBf16)))
        out[Key{(int64_t)N, (int64_t)K, (int64_t)NL, (int64_t)Sd, (int)prec, (int)fl}] = Entry{(int)v, ms};
    }
    pos = b + 1;
  }
  return out;
}

bool write_cache(const char* path, const std::map<Key, Entry>& m) {
  std::ofstream f(path);
  if (!f) return false;
  f << "{\"qfx_autotune\": 1, \"entries\": [\n";
  size_t i = 0;
  for (const auto& kv : m) {
    f << "  {\"N\": " << std::get<0>(kv.first) << ", \"K\": " << std::get<1>(kv.first)
      << ", \"NL\": " << std::get<2>(kv.first) << ", \"Sd\": " << std::get<3>(kv.first)
      << ", \"prec\": " << std::get<4>(kv.first) << ", \"tc_flags\": " << std::get<5>(kv.first)
      << ", \"variant\": " << kv.second.variant << ", \"ms\": " << kv.second.ms << "}"
      << (++i < m.size() ? ",\n" : "\n");
  }
  f << "]}\n";
  return (bool)f;
}

}  // namespace

int tc_variant_of(int precision) {
  return precision == QFX_PREC_C3M_BF16X3   ? kVariantTcBf16
         : precision == QFX_PREC_C3M_BF16X2 ? kVariantTcBf16x2
                                            : kVariantTcTf32;
}

void apply_autotune_cache(qfx_plan* p, const char* path) {
  const auto m = read_cache(path);
  if (m.empty()) return;
  for (size_t i = 1; i < p->steps.size(); ++i) {
    Step& s = p->steps[i];
    auto it = m.find(Key{s.N, s.K, s.NL, s.Sd, p->precision, p->tc_flags});
    if (it == m.end()) continue;
    const int v = it->second.variant;
    if (v >= 10) {   // the tensor-core kernel
      if (p->precision != QFX_PREC_FP32_SIMT && tc_eligible(p->precision, s.K, s.N, s.P * s.Sd, p->tc_flags))
        s.variant = tc_variant_of(p->precision);
      continue;
    }
    if (v < 5 && (s.Sd % 2)) continue;
    s.variant = v;
  }
}

}  // namespace qfx

using namespace qfx;

extern "C" qfx_status qfx_autotune(const qfx_plan* p, const char* cache_path, void* workspace,
                                   size_t ws_bytes, void* stream) {
  if (!p || !cache_path || !workspace) return fail(QFX_EINVAL, "qfx_autotune: NULL argument");
  if ((uintptr_t)workspace & 255) return fail(QFX_EINVAL, "qfx_autotune: workspace not 256-byte aligned");
  auto cache = read_cache(cache_path);
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(QFX_ECUDA, "qfx_autotune: cudaEventCreate");
  qfx_status result = QFX_OK;
  char* ws = (char*)workspace;
  for (size_t i = 1; i < p->steps.size() && result == QFX_OK; ++i) {
    const Step& s = p->steps[i];
    const Key key{s.N, s.K, s.NL, s.Sd, p->precision, p->tc_flags};
    if (cache.count(key)) continue;
    const bool tc_ok = p->precision != QFX_PREC_FP32_SIMT &&
                       tc_eligible(p->precision, s.K, s.N, s.P * s.Sd, p->tc_flags);
    // operands in the workspace: S | site image (tensor-core candidate) | B | C, shrinking
    // the problem to fit
    const uint64_t img = tc_ok ? ((tc_scratch_bytes(p->precision, s.K, s.N) + 255) & ~255ull) : 0;
    const uint64_t sb = (((uint64_t)s.K * s.N * 8 + 255) & ~255ull) + img;
    int64_t P = s.P, Sd = s.Sd;
    auto need = [&](int64_t P_, int64_t Sd_) {
      return sb + (((uint64_t)P_ * s.K * Sd_ * 8 + 255) & ~255ull) + (uint64_t)P_ * s.N * Sd_ * 8;
    };
    while (need(P, Sd) > ws_bytes && P > 1) P = (P + 1) / 2;
    while (need(P, Sd) > ws_bytes && Sd > 2) Sd = (Sd / 2) + (Sd % 2);   // keeps Sd's parity class
    if (need(P, Sd) > ws_bytes) { result = fail(QFX_ENOMEM, "qfx_autotune: workspace too small"); break; }
    const char* S = ws;
    char* image = ws + (sb - img);
    const char* B = ws + sb;
    char* C = ws + sb + (((uint64_t)P * s.K * Sd * 8 + 255) & ~255ull);
    cudaMemsetAsync(ws, 0, need(P, Sd), st);
    Entry best{-1, 1e30};
    for (int v = 0; v < 10; ++v) {
      if (v < 5 && (Sd % 2)) continue;
      int err = launch_step(S, 0, B, 0, C, 0, P, s.K, s.N, s.NL, Sd, 1, v, QFX_PREC_FP32_SIMT, st);
      if (err) continue;   // a variant that does not launch for this shape is skipped
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3; ++r) launch_step(S, 0, B, 0, C, 0, P, s.K, s.N, s.NL, Sd, 1, v, QFX_PREC_FP32_SIMT, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) { result = fail(QFX_ECUDA, "qfx_autotune: timing"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double per = ms / 3.0 * ((double)s.P * s.Sd) / ((double)P * Sd);   // scaled to the full step
      if (per < best.ms) best = Entry{v, per};
    }
    // the tensor-core kernel needs P * Sd >= 128 in the shrunk problem too
    if (tc_ok && result == QFX_OK && tc_eligible(p->precision, s.K, s.N, P * Sd, p->tc_flags)) {
      int err = launch_step_tc(S, 0, B, 0, C, 0, P, s.K, s.N, s.NL, Sd, 1, p->precision, image, 0, st,
                               p->tc_flags);
      if (!err) {
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r)
          launch_step_tc(S, 0, B, 0, C, 0, P, s.K, s.N, s.NL, Sd, 1, p->precision, image, 0, st, p->tc_flags);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { result = fail(QFX_ECUDA, "qfx_autotune: timing"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / 3.0 * ((double)s.P * s.Sd) / ((double)P * Sd);
        if (per < best.ms) best = Entry{kVariantTcBf16, per};
      }
    }
    if (best.variant >= 0) cache[key] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != QFX_OK) return result;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "qfx_autotune");
  if (!write_cache(cache_path, cache)) return fail(QFX_EINVAL, "qfx_autotune: cannot write the cache file");
  return QFX_OK;
}
