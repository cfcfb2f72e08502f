// The device-resident graph behind an opmos_graph handle (host-side view).
#pragma once

#include <cstdint>

#include "opmos_dev.cuh"

struct opmos_graph {
  uint32_t n = 0, d = 0, maxdeg = 0;
  uint64_t m = 0;
  uint32_t *rowptr = nullptr, *col = nullptr, *cost = nullptr;
  uint32_t *rrowptr = nullptr, *rsrc = nullptr, *rcost = nullptr;
  uint32_t* delta = nullptr;  // per objective, device
  opmos::GraphDev dev{};
};
