// Internal structures of the qtensor library (host side and launch descriptors).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qtensor.h"

namespace qt {

// ---------------------------------------------------------------------------
// Network (Sec. IV.A-B): tensors over binary indices, FP64 data.
// ---------------------------------------------------------------------------
struct Tensor {
  std::vector<int32_t> labels;  // axis t of the data is labels[t] (bit t of the element index)
  std::vector<double> data;     // interleaved (re, im), 2 * 2^rank doubles
};

// ---------------------------------------------------------------------------
// Line graph as dense bitset rows (Sec. IV.B) and greedy ordering (Sec. V.A.1).
// ---------------------------------------------------------------------------
struct BitGraph {
  int n = 0;  // vertices
  int W = 0;  // 64-bit words per row
  std::vector<uint64_t> rows;
  std::vector<uint8_t> alive;
  std::vector<uint8_t> keep;  // open indices (Sec. VII): never eliminated nor sliced; empty = none

  // an alive vertex that an order or a slicing round may take
  bool takeable(int v) const { return alive[v] && (keep.empty() || !keep[v]); }

  void init(int nv);
  uint64_t* row(int v) { return rows.data() + (size_t)v * W; }
  const uint64_t* row(int v) const { return rows.data() + (size_t)v * W; }
  bool has(int a, int b) const { return (row(a)[b >> 6] >> (b & 63)) & 1u; }
  void add_edge(int a, int b);
  int degree(int v) const;
  // joins v's neighbours into a clique and deletes v; returns v's neighbour count
  int eliminate(int v);
  // deletes v without joining its neighbours (slicing)
  void remove(int v);
};

struct OrderResult {
  std::vector<int32_t> order;
  std::vector<int32_t> widths;
};

OrderResult greedy_order(const BitGraph& g, int algo);
// randomised greedy (Sec. V.A.2): best of q Boltzmann-weighted eliminations
OrderResult rgreedy_order(const BitGraph& g, double tau, int q, uint64_t seed);

struct SlicePlan {
  std::vector<int32_t> order;   // every non-sliced vertex, elimination order
  std::vector<int32_t> widths;  // neighbour count of each step of `order` as planned
  std::vector<int32_t> sliced;  // sliced vertices, slice-bit order
  int32_t slice_step = 0;       // first round's step s_1 (0 without slicing)
  int32_t width = 0;
  int64_t greedy_runs = 0;      // ordering runs the search made
};

SlicePlan step_dependent_slicing(const BitGraph& g, int algo, int width_limit, int max_vars,
                                 int r);

BitGraph line_graph(const std::vector<Tensor>& tensors, int n_vars);

// ---------------------------------------------------------------------------
// Compiled schedule.
// ---------------------------------------------------------------------------
enum TensorKind { TK_GATE = 0, TK_PREFIX = 1, TK_SLICE = 2 };

struct STensor {
  int kind = TK_GATE;
  int gate = -1;                // index into the network's tensors for TK_GATE
  std::vector<int32_t> labels;  // canonical: ascending position (sliced labels on top)
  int rank = 0;                 // number of labels (sliced included)
  int nsliced = 0;              // labels that are sliced vertices
  uint64_t smask = 0;           // slice-id bits present (bit j: j-th sliced vertex)
  int64_t offset = 0;           // element offset inside its region
  int64_t meta = 0;             // meta slot (shared) or first slot (per slice)
  int producer = -1;            // step that writes it (-1 for gates)
  int last_use = -1;            // last step (then group) that reads it
  bool virt = false;            // produced and consumed inside one fused group: never stored
};

struct SStep {
  int region = 1;               // 0 prefix (once, unsliced), 1 per slice
  int var = -1;                 // bucket variable
  std::vector<int32_t> ops;     // schedule tensor ids
  std::vector<int32_t> ulabels; // union labels as the step sees them (canonical order)
  int out = -1;                 // schedule tensor id of the result
  int u = 0, c = 0, nsum = 1;
  int64_t flops = 0, bytes = 0;
};

// A launch: consecutive bucket steps fused when the indices they sum out die
// together. Step i+l of the group (l = 1..nsum-1) adds operands whose indices
// all lie in the first step's union U; they enter at "level" l, i.e. after the
// l lowest U bits have been summed, so the arithmetic is exactly that of the
// separate steps while the intermediate results never reach memory.
struct SGroup {
  int region = 1;
  int first = 0, nsteps = 1;     // steps first .. first + nsteps - 1
  std::vector<int32_t> ops;      // tensor ids, level 0 first
  std::vector<int32_t> levels;   // level of each operand
  std::vector<int32_t> ulabels;  // U of the first step (canonical order)
  int out = -1;                  // result of the last step
  int u = 0, nsum = 1, c = 0;
  int64_t flops = 0, bytes = 0;  // flops: sum over the steps; bytes: operands once + result
  // GEMM form (complex precisions only): with A and B the two largest operands and
  // every other operand's indices inside A or inside B, the launch is
  //   out[bt][m][n] = sum_k A'[bt][m][k] B'[bt][n][k]
  // A' = A times the operands folded into it, summed over the summed indices only A
  // has (B' likewise); k: summed indices both have; m, n: output indices of A only,
  // B only; bt: output indices of both. Masks are over the group's U bits.
  bool gemm = false;
  int gA = -1, gB = -1;              // indices into ops
  std::vector<int8_t> side;          // per operand: 0 folded into A', 1 into B'
  uint32_t mK = 0, mSA = 0, mSB = 0, mM = 0, mN = 0, mBt = 0;
  int64_t scratch_a = 0, scratch_b = 0;  // arena offsets of A', B' (planar re | im)
  // Triangle form (complex precisions): three large operands A, B, C and every
  // summed index in exactly two of them -- class K (A and B), X (A and C), Y (B and
  // C); the other operands lie inside C (folded into C) or are summed-only inside
  // K (a weight over K). Then out = sum_k w(k) sum_x A[k,x] sum_y B[k,y] C[x,y].
  bool tri = false;
  int tA = -1, tB = -1, tC = -1;     // indices into ops
  uint32_t tK = 0, tX = 0, tY = 0;   // summed U bits of each class
  std::vector<int8_t> tfold;         // per operand: 0 large, 1 folded into C, 2 weight over K
  int tCbits = 0;                    // indices of C (its folded copy C' has 2^tCbits elements)
  int64_t scratch_t = 0;             // arena offset of C'
};

struct Schedule {
  bool valid = false;
  bool force_gemm = false;       // copy of the network option at compile time
  bool force_stream = false;     // copy of the network option at compile time
  bool force_tri = false;        // copy of the network option at compile time
  int tma_block = 0;             // copy of the network option at compile time
  int tcgen05 = 0;               // copy of the network option at compile time
  bool force_scaled = false;     // copy of the network option at compile time
  bool fused = true;             // steps grouped into fused launches
  uint64_t generation = 0;      // changes with every compile
  int precision = QT_FP32_SIMT;
  int elem_bytes = 8;
  int k = 0;
  int n_open = 0;                // open indices: the result has 2^n_open amplitudes
  int64_t n_amps = 1;
  int64_t nslices = 1;
  int64_t batch = 1;
  std::vector<int32_t> pos;     // variable -> canonical position
  std::vector<STensor> tensors;
  std::vector<SStep> steps;
  std::vector<SGroup> groups;
  int n_prefix_steps = 0;
  std::vector<int32_t> scalars; // tensors whose value multiplies the slice result
  // region sizes in elements
  int64_t gate_elems = 0, prefix_elems = 0, slice_elems = 0;
  int64_t n_shared_meta = 0, n_slice_meta_tensors = 0;
  // workspace layout (bytes)
  size_t off_gates = 0, off_prefix = 0, off_slices = 0, off_meta = 0, off_partials = 0,
         off_acc = 0, off_terms = 0, off_segtab = 0, off_err = 0, total_bytes = 0;
  // ledger
  int64_t prefix_flops = 0, prefix_bytes = 0, slice_flops = 0, slice_bytes = 0;
  int64_t prefix_launch_bytes = 0, slice_launch_bytes = 0;  // bytes of the (fused) launches
  int prefix_width = 0, slice_width = 0;
};

constexpr int kMaxFusedSum = 6;   // indices summed by one launch
constexpr int kMaxGroupOps = 12;  // operands of one launch

// The last n_open variable ids are open indices (Sec. VII): never summed, they
// index the result.
bool compile_schedule(const std::vector<Tensor>& net, int n_vars, const SlicePlan& plan,
                      int precision, int64_t batch, bool fuse, Schedule& out, std::string& err,
                      int n_open = 0);

std::string schedule_json(const Schedule& s, const SlicePlan& plan);

constexpr size_t kScalarTermBytes = 40;  // device ScalarTerm record
constexpr size_t kStepRecordBytes = 2048;  // segment-table bytes reserved per launch group

// Canonical-layout copy of a gate tensor's data (FP64 interleaved).
std::vector<double> canonical_data(const Tensor& t, const std::vector<int32_t>& canon_labels);

// One profiled kernel launch (events recorded around it on the caller's stream).
struct ProfRec {
  int step;         // schedule step (-1: finalize/reduce)
  int kernel;       // 0 flat bucket, 1 tiled bucket, 2 finalize + reduce
  int64_t slices;   // slices processed by the launch
  int64_t bytes;    // algorithmic bytes of the launch (ledger bytes x slices)
  int64_t flops;    // ledger flops of the launch
  void* ev0;
  void* ev1;
};

// learned proposals (learn.cpp)
constexpr int kProposalFeatures = 16;
int mlp_param_count(int nf, int hidden);
void mlp_forward_host(const float* params, int nf, int hidden, const float* x, int batch, float* y);

}  // namespace qt

// The opaque network handle.
struct qt_net {
  int32_t n = 0, p = 0, n_edges = 0, n_vars = 0;
  std::vector<int32_t> edges;
  std::vector<double> gammas, betas;
  std::vector<uint8_t> z;
  std::vector<int32_t> open;     // open qubits (Sec. VII); open j is variable n*p + j
  std::vector<qt::Tensor> tensors;
  bool ordered = false;
  int algo = QT_GREEDY_MINFILL;
  qt::SlicePlan plan;
  qt::Schedule sched;
  // host staging of the canonical gate data for the prepared precision
  std::vector<unsigned char> gate_stage;
  std::vector<unsigned char> meta_stage;
  bool stage_dirty = true;
  // what qt_upload last copied: the schedule generation, the gate data version (bumped
  // by every change of angles or bitstring) and the workspace it went to
  uint64_t data_version = 1;
  uint64_t uploaded_gen = 0, uploaded_data = 0;
  const void* uploaded_ws = nullptr;
  // tracing: CUDA events around every launch when enabled
  bool prof = false;
  std::vector<qt::ProfRec> prof_recs;
  std::vector<void*> prof_pool;  // recycled cudaEvent_t
  int64_t launches = 0;          // kernel launches issued by this network
  bool graphs = true;            // replay runs as captured CUDA graphs
  bool fuse = true;              // fuse bucket steps whose summed indices die together
  bool force_gemm = false;       // GEMM-form launches by default also in FP32 mode
  bool force_stream = false;     // ... with the streaming kernel where it applies
  bool segments = true;          // runs of small launches as one segment launch
  int seg_max_u = 12;            // union indices of a step a segment may hold (at most 13)
  int seg_cluster = 0;           // blocks per slice of a segment launch: 0 chosen, 1, 2, 4, 8
  bool concurrent = true;        // captured graphs run independent slice launches concurrently
  bool force_tri = false;        // triangle-form launches by default where they apply
  bool tma = true;               // tiled GEMM stages its blocks with tensor copies (TMA)
  int64_t tma_launches = 0;      // tiled GEMM launches that took the tensor-copy staging
  int tma_block = 0;             // tiled GEMM register block: 0 chosen, 1 2 x 2, 2 / 3 wide
  int64_t stream_launches = 0;   // GEMM-form launches by the streaming kernel
  int tcgen05 = 0;               // GEMM form on tcgen05: 0 default + autotuned, 1 forced, 2 never
  int64_t umma_launches = 0;     // GEMM-form launches by the tcgen05 kernel
  bool force_scaled = false;     // the tiled kernel always takes its scaled path
  void* engine = nullptr;        // engine.cu: launch descriptors and graph cache
  ~qt_net();
};

namespace qt {
// Prepares `net` in `precision` with the largest slice batch whose workspace size plus
// room() bytes is at most `budget` (room() is evaluated on the batch-1 schedule). Returns
// QT_ENOMEM, with both sizes in `err`, when one slice does not fit; prepare errors as
// qt_prepare (message in qt_last_error()).
qt_status prepare_fitting(qt_net* net, int32_t precision, size_t budget, size_t (*room)(const qt_net*, const void*),
                          const void* room_arg, std::string& err);
// The engine's launch descriptors, autotuned choices and captured graph: taken out of the
// network (which then builds a fresh cache on its next run) and put back, the fresh one
// deleted.
void* engine_detach(qt_net* net);
void engine_restore(qt_net* net, void* saved);
// Line graph of the network plus the clique on its open indices (Sec. VII: the
// result tensor over them), those indices marked as kept.
BitGraph network_graph(const qt_net* net);
}  // namespace qt
