// Internal structures of the batched lightcone energy.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "qt_internal.h"

namespace qt {

// one edge's lightcone network, its order and its compiled schedule
struct EnergyNet {
  std::vector<Tensor> tensors;
  // per tensor: how its data follows from the angles (angle sweeps rebuild the gate
  // data without re-planning): kind (0 constant, 1 phase of layer k, 2 mixer of
  // layer k) | layer k << 4 | side << 12 (1 ket, 2 bra)
  std::vector<int32_t> tags;
  int n_vars = 0;
  double norm = 1.0;  // 2^(-|S|)
  SlicePlan plan;
  Schedule sched;
};

// device tables (plain data, uploaded as is)
struct EOp {
  uint32_t off;       // element offset: in the gate region, or in the block's arena
  uint32_t umask;     // U bits of the operand
  uint16_t level;     // nested-sum level
  uint16_t in_arena;  // 1: offset is in the block's arena
};
struct EStep {
  uint16_t m, u, nsum, pad;
  uint32_t first_op;  // index into the operand table
  uint32_t out;       // arena offset of the result
};
struct ENet {
  uint32_t first_step, nsteps, first_scalar, nscalars;
  uint32_t edge, pad;
  double norm;
};

}  // namespace qt

struct qt_energy {
  int32_t n = 0, p = 0, algo = 0;
  std::vector<int32_t> edges;
  std::vector<std::vector<int>> adj;
  std::vector<double> gammas, betas;
  std::vector<qt::EnergyNet> nets;
  bool fuse = true;
  bool compiled = false;
  int precision = 0, elem_bytes = 8;
  // packed tables
  std::vector<qt::EOp> h_ops;
  std::vector<qt::EStep> h_steps;
  std::vector<qt::ENet> h_nets;
  std::vector<uint32_t> h_scalars;
  std::vector<unsigned char> h_gates;
  int64_t gate_elems = 0, arena_elems = 0;
  int64_t total_flops = 0, total_bytes = 0;
  int max_width = 0;
  std::vector<int> hist_width;
  // launch shape (autotuned) and workspace layout
  int block_threads = 128;
  int blocks = 0;
  size_t off_gates = 0, off_ops = 0, off_steps = 0, off_nets = 0, off_scalars = 0,
         off_arenas = 0, off_zz = 0, off_counter = 0, total_bytes_ws = 0;
  void* engine = nullptr;  // graph cache
  // angle sweep: workspace layout for sweep_sets angle sets, staged gate images
  int sweep_sets = 0;
  size_t sw_off_gates = 0, sw_off_ops = 0, sw_off_steps = 0, sw_off_nets = 0, sw_off_scalars = 0,
         sw_off_zz = 0, sw_off_energy = 0, sw_off_counter = 0, sw_off_arenas = 0, sw_total = 0;
  // the sweep's gate images are assembled on the device: one image with every
  // angle-free tensor in place (the template), the angle-dependent gates' element
  // offsets and codes (kind | layer << 4 | side << 12), and per set a table of their
  // entries (cos and sin of the set's angles, FP64 on the host, cast)
  std::vector<unsigned char> sw_template;
  std::vector<uint32_t> sw_slots, sw_codes;
  std::vector<unsigned char> sw_table;
  size_t sw_off_tmpl = 0, sw_off_slots = 0, sw_off_codes = 0, sw_off_table = 0;
  const void* sw_tmpl_ws = nullptr;  // workspace holding the template and slot lists
  ~qt_energy();
};

namespace qt {
bool energy_build_networks(qt_energy* E, std::string& err);
bool energy_compile(qt_energy* E, int precision, std::string& err);
// gate data of every network for one angle set, in the compiled precision and layout
void energy_gate_image(const qt_energy* E, const double* gammas, const double* betas,
                       unsigned char* dst);
// the sweep's template image and angle-dependent gate slots (see qt_energy)
void energy_sweep_template(qt_energy* E);
// per set, per layer k: phase (re, im) and mixer (cos, sin) for ket side 1 and bra side 2,
// 8 values [kind][side][2] in the compiled precision
void energy_sweep_table(qt_energy* E, int n_sets, const double* gammas, const double* betas);
}  // namespace qt
