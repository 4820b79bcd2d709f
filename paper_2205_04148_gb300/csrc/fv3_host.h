// fv3_host.h -- host-side structures of the FV3 substep library (internal).
#pragma once
#include <vector>

#include "fv3_dev.cuh"

namespace fv3 {

enum PlanKind { K_CELL3 = 0, K_CELL1, K_DGRID, K_CGRID, K_LENGTH, K_COSINE, K_NUM };

struct Plans {
  std::vector<HaloEntry> p[K_NUM];
};

struct GridSpec {
  bool cubed;
  double dx, radius, omega;
};

struct HostMetric {
  std::vector<double> area, rarea, fA;
  std::vector<double> dx, rdx, dyc, rdyc, cosy, siny;
  std::vector<double> dy, rdy, dxc, rdxc, cosx, sinx;
  std::vector<double> fC, rareac;
  double da_min = 0;
};

void build_metric(const GridSpec& spec, int m, const Geo& g, HostMetric& M, Plans& plans);

}  // namespace fv3
