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
};

namespace sbh {
void set_error(const std::string& msg);
}
