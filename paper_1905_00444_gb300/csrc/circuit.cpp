// Circuit ingest and validation (the RQC class of Sec. III: planar grid, two-qubit
// gates only between grid neighbours) and the project's text format.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <sstream>
#include <string>
#include <vector>

#include "qfx_internal.h"

namespace {

bool two_qubit_kind(int kind) {
  return kind == QFX_GATE_CZ || kind == QFX_GATE_U2 || kind == QFX_GATE_U4;
}

// matrix values a kind carries: 32 for a general two-qubit gate, 8 otherwise
int mat_values(int kind) { return kind == QFX_GATE_U4 ? 32 : 8; }

bool neighbours(int rows, int cols, int a, int b) {
  int ra = a / cols, ca = a % cols, rb = b / cols, cb = b % cols;
  return (ra == rb && std::abs(ca - cb) == 1) || (ca == cb && std::abs(ra - rb) == 1);
}

qfx_status build(int32_t rows, int32_t cols, const qfx_gate* gates, int64_t n_gates,
                 qfx_circuit** out) {
  if (!out) return qfx::fail(QFX_EINVAL, "qfx_circuit_create: out is NULL");
  *out = nullptr;
  if (rows < 1 || cols < 1 || (int64_t)rows * cols > qfx::kMaxSites)
    return qfx::fail(QFX_EINVAL, "qfx_circuit_create: need 1 <= rows*cols <= " + std::to_string(qfx::kMaxSites));
  if (n_gates < 0 || (n_gates > 0 && !gates))
    return qfx::fail(QFX_EINVAL, "qfx_circuit_create: bad gate array");
  const int n = rows * cols;
  auto* c = new qfx_circuit;
  c->rows = rows;
  c->cols = cols;
  c->gates.reserve((size_t)n_gates);
  for (int64_t i = 0; i < n_gates; ++i) {
    const qfx_gate& g = gates[i];
    std::string where = "gate " + std::to_string(i) + ": ";
    if (g.layer < 0) { delete c; return qfx::fail(QFX_EINVAL, where + "negative layer"); }
    if (g.q0 < 0 || g.q0 >= n) { delete c; return qfx::fail(QFX_EINVAL, where + "q0 out of range"); }
    if (g.q1 >= n || g.q1 < -1) { delete c; return qfx::fail(QFX_EINVAL, where + "q1 out of range"); }
    if (g.q1 >= 0) {
      if (g.q1 == g.q0) { delete c; return qfx::fail(QFX_EINVAL, where + "q0 == q1"); }
      if (!neighbours(rows, cols, g.q0, g.q1)) {
        delete c;
        return qfx::fail(QFX_EINVAL, where + "two-qubit gate between non-neighbours");
      }
    }
    if (g.kind < QFX_GATE_H || g.kind > QFX_GATE_U4) {
      delete c;
      return qfx::fail(QFX_EINVAL, where + "unknown kind");
    }
    bool two = g.q1 >= 0;
    if (two != two_qubit_kind(g.kind)) { delete c; return qfx::fail(QFX_EINVAL, where + "kind does not match arity"); }
    const int nv = mat_values(g.kind);
    for (int k = 0; k < nv; ++k)
      if (!std::isfinite(g.mat[k])) { delete c; return qfx::fail(QFX_EINVAL, where + "non-finite matrix entry"); }
    qfx::Gate q{g.layer, g.q0, g.q1, g.kind, {}, (int)i};
    std::memcpy(q.m, g.mat, sizeof(double) * nv);
    c->gates.push_back(q);
  }
  std::stable_sort(c->gates.begin(), c->gates.end(),
                   [](const qfx::Gate& a, const qfx::Gate& b) { return a.layer < b.layer; });
  // disjoint qubits within each layer
  for (size_t i = 0; i < c->gates.size();) {
    size_t j = i;
    std::vector<char> used((size_t)n, 0);
    while (j < c->gates.size() && c->gates[j].layer == c->gates[i].layer) {
      const auto& g = c->gates[j];
      if (used[g.q0] || (g.q1 >= 0 && used[g.q1])) {
        int layer = g.layer;
        delete c;
        return qfx::fail(QFX_EINVAL, "layer " + std::to_string(layer) + ": qubit used twice");
      }
      used[g.q0] = 1;
      if (g.q1 >= 0) used[g.q1] = 1;
      ++j;
    }
    i = j;
  }
  *out = c;
  return QFX_OK;
}

int kind_from_name(const std::string& s) {
  static const char* names[] = {"H", "SQRT_X", "SQRT_Y", "T", "CZ", "U1", "U2", "U4"};
  for (int i = 0; i < 8; ++i)
    if (s == names[i]) return i;
  return -1;
}

}  // namespace

extern "C" qfx_status qfx_circuit_create(int32_t rows, int32_t cols, const qfx_gate* gates,
                                         int64_t n_gates, qfx_circuit** out) {
  try {
    return build(rows, cols, gates, n_gates, out);
  } catch (...) {
    return qfx::fail(QFX_EINVAL, "qfx_circuit_create: internal error");
  }
}

extern "C" qfx_status qfx_circuit_from_text(const char* text, qfx_circuit** out) {
  if (!text || !out) return qfx::fail(QFX_EINVAL, "qfx_circuit_from_text: NULL argument");
  try {
    std::istringstream in(text);
    std::string line;
    int rows = -1, cols = -1, lineno = 0;
    std::vector<qfx_gate> gates;
    while (std::getline(in, line)) {
      ++lineno;
      auto hash = line.find('#');
      if (hash != std::string::npos) line.resize(hash);
      std::istringstream ls(line);
      std::string first;
      if (!(ls >> first)) continue;
      std::string where = "line " + std::to_string(lineno) + ": ";
      if (first == "grid") {
        if (!(ls >> rows >> cols)) return qfx::fail(QFX_EINVAL, where + "bad grid line");
        continue;
      }
      if (rows < 0) return qfx::fail(QFX_EINVAL, where + "gate before the grid line");
      qfx_gate g{};
      try {
        g.layer = std::stoi(first);
      } catch (...) {
        return qfx::fail(QFX_EINVAL, where + "bad layer");
      }
      std::string kname;
      if (!(ls >> kname)) return qfx::fail(QFX_EINVAL, where + "missing kind");
      g.kind = kind_from_name(kname);
      if (g.kind < 0) return qfx::fail(QFX_EINVAL, where + "unknown kind " + kname);
      bool two = two_qubit_kind(g.kind);
      if (!(ls >> g.q0)) return qfx::fail(QFX_EINVAL, where + "missing q0");
      g.q1 = -1;
      if (two && !(ls >> g.q1)) return qfx::fail(QFX_EINVAL, where + "missing q1");
      const int nv = mat_values(g.kind);
      for (int k = 0; k < nv; ++k)
        if (!(ls >> g.mat[k]))
          return qfx::fail(QFX_EINVAL, where + "need " + std::to_string(nv) + " matrix values");
      std::string extra;
      if (ls >> extra) return qfx::fail(QFX_EINVAL, where + "trailing text");
      gates.push_back(g);
    }
    if (rows < 0) return qfx::fail(QFX_EINVAL, "qfx_circuit_from_text: no grid line");
    return build(rows, cols, gates.data(), (int64_t)gates.size(), out);
  } catch (...) {
    return qfx::fail(QFX_EINVAL, "qfx_circuit_from_text: internal error");
  }
}

extern "C" void qfx_circuit_destroy(qfx_circuit* c) { delete c; }
