// Host-side plan of a joint-cut HSF simulation (internal).
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hsf.h"
#include "common.h"

namespace hsf {

using cd = std::complex<double>;

struct GateH {
  int kind = 0;
  int nq = 0;
  int q[4] = {0, 0, 0, 0};
  double param = 0.0;
  int param_id = -1;
  std::vector<cd> m;       // 2^nq x 2^nq, row-major
  bool diag = false;
  int side = 0;            // 0 = a (all qubits > l), 1 = b (all <= l), 2 = crossing
};

struct BlockH {
  std::vector<int> gates;  // circuit order
  std::vector<int> qubits; // descending: a-qubits first
  std::vector<int> qa, qb; // descending
  int rank = 0;
  std::vector<double> sigma;
  std::vector<cd> x, y;    // rank x 4^ka and rank x 4^kb, sqrt(sigma) folded in
};

// One op of a side program, on side-local logical qubits (q[0] = matrix MSB).
struct OpH {
  int type = OP_DENSE;
  int nq = 0;
  int q[3] = {0, 0, 0};
  std::vector<cd> m;       // dense: 4^nq per digit; diag: 2^nq per digit
  int digits = 1;          // > 1: Schmidt factor, matrices for every digit
  int block = -1;
};

struct PassH {
  uint64_t active = 0;     // storage bits in the tile
  int t = 0;
  std::vector<OpH> ops;
  // device
  size_t ops_off = 0, mats_off = 0;   // byte offsets in the device table
  int num_ops = 0;
};

struct LevelH {
  std::vector<OpH> ops;
  std::vector<PassH> passes;
};

struct SideH {
  int h = 0;
  int offset = 0;          // global qubit of local qubit 0
  std::vector<LevelH> levels;   // 0 .. B
};

}  // namespace hsf

struct hsf_plan {
  int n = 0, cut = 0, na = 0, nb = 0;
  int precision = 0, gemm_mode = 0, flags = 0, tile_max = 14;
  double rank_tol = 1e-12;
  uint64_t max_paths = 0;
  std::vector<hsf::GateH> gates;
  std::vector<hsf::BlockH> blocks;
  std::vector<uint64_t> radix;      // radix[k] = rank of level k (radix[0] = 1), k = 0..B
  std::vector<uint64_t> below;      // below[k] = product of radix[k+1..B] (subtree leaves)
  uint64_t num_paths = 1;
  hsf::SideH side[2];               // 0 = a, 1 = b
  void *dev_table = nullptr;        // ops + matrices of every pass
  size_t dev_table_bytes = 0;
  int64_t tree_nodes = 0;
  int64_t launches = 0;
  struct ProfRec { int kind; cudaEvent_t e0, e1; double bytes, flops; };
  std::vector<ProfRec> prof;
};
