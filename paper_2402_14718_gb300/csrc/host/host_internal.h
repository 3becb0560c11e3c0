// Internal host-side types of the event generator, QUBO builder and tracks.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "../../../include/sb.h"

struct sb_event {
  std::vector<int32_t> layer;
  std::vector<double> r, phi, z, x, y;
  std::vector<int32_t> particle;
  int32_t n_true = 0;
};

struct sb_qubo {
  int32_t n = 0;
  std::vector<int32_t> rowptr, col;
  std::vector<double> val, lin, quality, kappa, dtheta;
  std::vector<int8_t> cls;
  std::vector<int32_t> trip;  // 3 per triplet
  double w_c = 1.0;           // conflict weight the couplings were built with
  int32_t n_hits = 0;         // hits of the event (hit ids lie in [0, n_hits))
};

namespace sbh {
void set_error(const std::string& msg);
}
