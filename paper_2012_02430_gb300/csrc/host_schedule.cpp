// Schedule compiler: turns (network, order, slices) into the list of bucket
// steps the GPU executes, with canonical tensor layouts, memory offsets and
// the integer FLOP/byte ledger.
//
// Bucket elimination follows Alg. 1: bucket i holds the tensors whose earliest
// index (by elimination position) is the i-th vertex of the order; its tensors
// are multiplied over the union of their indices and that vertex is summed
// out; the result goes to the bucket of its own earliest index, or multiplies
// the result when it is a scalar. Slicing follows Alg. 1 and Eq. 2: steps
// before the first slice step run once on the unsliced network, later steps
// run once per slice with every sliced index fixed.
//
// Canonical layout: a tensor's indices are ordered by elimination position,
// earliest = least significant bit of the element index; sliced vertices get
// positions above every eliminated one (in slice-bit order), so fixing them
// selects one contiguous block of a shared tensor. In bucket i every operand
// has the bucket vertex as bit 0, so the two values that are summed are
// adjacent in memory.
#include <algorithm>
#include <cstdio>
#include <map>
#include <sstream>

#include "qt_internal.h"

namespace qt {

std::vector<double> canonical_data(const Tensor& t, const std::vector<int32_t>& canon) {
  const int r = (int)t.labels.size();
  std::vector<int> axis_of(r);  // canonical bit b -> axis of the gate data
  for (int b = 0; b < r; ++b)
    for (int a = 0; a < r; ++a)
      if (t.labels[a] == canon[b]) axis_of[b] = a;
  const size_t n = (size_t)1 << r;
  std::vector<double> out(2 * n);
  for (size_t e = 0; e < n; ++e) {
    size_t src = 0;
    for (int b = 0; b < r; ++b)
      if ((e >> b) & 1u) src |= (size_t)1 << axis_of[b];
    out[2 * e] = t.data[2 * src];
    out[2 * e + 1] = t.data[2 * src + 1];
  }
  return out;
}

namespace {

// First-fit allocator over an element range, for liveness-based reuse.
struct Arena {
  std::map<int64_t, int64_t> free_blocks;  // offset -> size
  int64_t top = 0;
  static int64_t align(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
  int64_t alloc(int64_t n, int64_t a) {
    n = align(n, a);
    for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
      if (it->second >= n) {
        int64_t off = it->first;
        int64_t rest = it->second - n;
        free_blocks.erase(it);
        if (rest > 0) free_blocks[off + n] = rest;
        return off;
      }
    }
    int64_t off = top;
    top += n;
    return off;
  }
  void release(int64_t off, int64_t n, int64_t a) {
    n = align(n, a);
    auto it = free_blocks.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_blocks.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_blocks.erase(nx);
    }
    if (it != free_blocks.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_blocks.erase(it);
      }
    }
  }
};

constexpr int64_t kArenaAlign = 64;  // elements (512 B for complex64)
constexpr int64_t kGateAlign = 2;    // elements: keeps every value pair 16-byte aligned

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

bool compile_schedule(const std::vector<Tensor>& net, int n_vars, const SlicePlan& plan,
                      int precision, int64_t batch, bool fuse, Schedule& S, std::string& err,
                      int n_open) {
  static uint64_t next_generation = 1;
  S = Schedule();
  S.fused = fuse;
  S.generation = next_generation++;
  S.precision = precision;
  S.elem_bytes = precision == QT_FP64 ? 16 : 8;
  const int n_order = (int)plan.order.size();
  S.k = (int)plan.sliced.size();
  S.nslices = (int64_t)1 << S.k;
  S.batch = std::max<int64_t>(1, std::min<int64_t>(batch, S.nslices));
  if (n_open < 0 || n_open > QT_MAX_OPEN || n_open > n_vars) {
    err = "bad number of open indices";
    return false;
  }
  S.n_open = n_open;
  S.n_amps = (int64_t)1 << n_open;
  S.pos.assign(n_vars, -1);
  std::vector<int> slice_bit(n_vars, -1), open_bit(n_vars, -1);
  for (int i = 0; i < n_order; ++i) S.pos[plan.order[i]] = i;
  // open indices sit above every eliminated one and below the sliced ones, so a
  // tensor left over the open (and sliced) indices is indexed (open bits, slice bits)
  for (int j = 0; j < n_open; ++j) {
    const int v = n_vars - n_open + j;
    if (S.pos[v] >= 0) {
      err = "an open index is in the elimination order";
      return false;
    }
    S.pos[v] = n_order + j;
    open_bit[v] = j;
  }
  for (int j = 0; j < S.k; ++j) {
    if (open_bit[plan.sliced[j]] >= 0) {
      err = "an open index is sliced";
      return false;
    }
    S.pos[plan.sliced[j]] = n_order + n_open + j;
    slice_bit[plan.sliced[j]] = j;
  }
  for (int v = 0; v < n_vars; ++v)
    if (S.pos[v] < 0) {
      err = "plan does not cover every variable";
      return false;
    }
  const int boundary = S.k > 0 ? plan.slice_step : 0;
  auto by_pos = [&](int32_t a, int32_t b) { return S.pos[a] < S.pos[b]; };

  std::vector<std::vector<int32_t>> buckets(n_order);
  auto place = [&](int32_t tid, int region_of_creation) {
    STensor& t = S.tensors[tid];
    int e = -1;
    for (int32_t l : t.labels)
      if (slice_bit[l] < 0 && open_bit[l] < 0 && (e < 0 || S.pos[l] < e)) e = S.pos[l];
    (void)region_of_creation;
    if (e < 0) {
      // only sliced and open indices left: a factor of the slice's result tensor
      S.scalars.push_back(tid);
    } else {
      buckets[e].push_back(tid);
    }
  };
  auto make_tensor = [&](int kind, std::vector<int32_t> labels) {
    STensor t;
    t.kind = kind;
    std::sort(labels.begin(), labels.end(), by_pos);
    t.labels = labels;
    t.rank = (int)labels.size();
    for (int32_t l : labels)
      if (slice_bit[l] >= 0) {
        t.nsliced++;
        t.smask |= 1ull << slice_bit[l];
      }
    S.tensors.push_back(t);
    return (int32_t)S.tensors.size() - 1;
  };
  for (size_t g = 0; g < net.size(); ++g) {
    int32_t tid = make_tensor(TK_GATE, net[g].labels);
    S.tensors[tid].gate = (int)g;
    place(tid, 0);
  }
  for (int i = 0; i < n_order; ++i) {
    std::vector<int32_t> bucket = buckets[i];
    if (bucket.empty()) continue;
    SStep st;
    st.region = i < boundary ? 0 : 1;
    st.var = plan.order[i];
    st.ops = bucket;
    std::vector<int32_t> uni;
    for (int32_t tid : bucket)
      for (int32_t l : S.tensors[tid].labels) {
        if (st.region == 1 && slice_bit[l] >= 0) continue;
        if (std::find(uni.begin(), uni.end(), l) == uni.end()) uni.push_back(l);
      }
    std::sort(uni.begin(), uni.end(), by_pos);
    if (uni.empty() || uni[0] != st.var) {
      err = "internal: bucket vertex is not the earliest index";
      return false;
    }
    st.ulabels = uni;
    st.u = (int)uni.size();
    st.c = st.u - 1;
    st.nsum = 1;
    if (st.c > 32 || st.u > 33) {
      err = "tensor rank above 32";
      return false;
    }
    std::vector<int32_t> out(uni.begin() + 1, uni.end());
    int32_t oid = make_tensor(st.region == 0 ? TK_PREFIX : TK_SLICE, out);
    S.tensors[oid].producer = (int)S.steps.size();
    st.out = oid;
    // ledger (Alg. 1 step, complex arithmetic)
    int64_t m = (int64_t)bucket.size();
    st.flops = 6 * (m - 1) * ((int64_t)1 << st.u) + 2 * (((int64_t)1 << st.u) - ((int64_t)1 << st.c));
    int64_t elems = (int64_t)1 << st.c;
    for (int32_t tid : bucket) {
      const STensor& t = S.tensors[tid];
      int rk = st.region == 1 ? t.rank - t.nsliced : t.rank;
      elems += (int64_t)1 << rk;
    }
    st.bytes = 8 * elems;
    for (int32_t tid : bucket) S.tensors[tid].last_use = (int)S.steps.size();
    S.steps.push_back(st);
    place(oid, st.region);
  }
  for (const SStep& st : S.steps) {
    if (st.region == 0) {
      S.n_prefix_steps++;
      S.prefix_flops += st.flops;
      S.prefix_bytes += st.bytes;
      S.prefix_width = std::max(S.prefix_width, st.c);
    } else {
      S.slice_flops += st.flops;
      S.slice_bytes += st.bytes;
      S.slice_width = std::max(S.slice_width, st.c);
    }
  }
  // launch groups: a step joins the previous group when its vertex is the next
  // position, it consumes the group's running result, every other operand lies
  // inside the group's U, and the limits on summed indices and operands hold
  auto seen_labels = [&](int32_t tid, int region) {
    std::vector<int32_t> out;
    for (int32_t l : S.tensors[tid].labels)
      if (region == 0 || slice_bit[l] < 0) out.push_back(l);
    return out;
  };
  for (int si = 0; si < (int)S.steps.size(); ++si) {
    const SStep& st = S.steps[si];
    bool joined = false;
    if (fuse && !S.groups.empty()) {
      SGroup& g = S.groups.back();
      const SStep& last = S.steps[g.first + g.nsteps - 1];
      bool ok = st.region == g.region && S.pos[st.var] == S.pos[last.var] + 1 &&
                g.nsum + 1 <= kMaxFusedSum;
      int nothers = 0;
      bool has_prev = false;
      if (ok) {
        for (int32_t tid : st.ops) {
          if (tid == last.out) {
            has_prev = true;
            continue;
          }
          ++nothers;
          for (int32_t l : seen_labels(tid, st.region))
            if (std::find(g.ulabels.begin(), g.ulabels.end(), l) == g.ulabels.end()) ok = false;
        }
      }
      ok = ok && has_prev && (int)g.ops.size() + nothers <= kMaxGroupOps;
      if (ok) {
        for (int32_t tid : st.ops)
          if (tid != last.out) {
            g.ops.push_back(tid);
            g.levels.push_back(g.nsum);
          }
        S.tensors[last.out].virt = true;
        g.nsteps++;
        g.nsum++;
        g.c = g.u - g.nsum;
        g.out = st.out;
        g.flops += st.flops;
        joined = true;
      }
    }
    if (!joined) {
      SGroup g;
      g.region = st.region;
      g.first = si;
      g.ops = st.ops;
      g.levels.assign(st.ops.size(), 0);
      g.ulabels = st.ulabels;
      g.out = st.out;
      g.u = st.u;
      g.nsum = 1;
      g.c = st.c;
      g.flops = st.flops;
      S.groups.push_back(g);
    }
  }
  for (SGroup& g : S.groups) {
    int64_t elems = (int64_t)1 << g.c;
    for (int32_t tid : g.ops) elems += (int64_t)1 << seen_labels(tid, g.region).size();
    g.bytes = 8 * elems;
    (g.region == 0 ? S.prefix_launch_bytes : S.slice_launch_bytes) += g.bytes;
  }
  // GEMM form of large groups (complex64 precisions)
  if (precision != QT_FP64) {
    for (SGroup& g : S.groups) {
      if (g.u < 14 || g.ops.size() < 2) continue;
      std::vector<uint32_t> mask(g.ops.size(), 0u);
      for (size_t j = 0; j < g.ops.size(); ++j)
        for (int32_t l : seen_labels(g.ops[j], g.region))
          for (int b = 0; b < g.u; ++b)
            if (g.ulabels[b] == l) mask[j] |= 1u << b;
      int a = -1, bb = -1;
      for (int j = 0; j < (int)g.ops.size(); ++j) {
        const int pj = __builtin_popcount(mask[j]);
        if (a < 0 || pj > __builtin_popcount(mask[a])) {
          bb = a;
          a = j;
        } else if (bb < 0 || pj > __builtin_popcount(mask[bb])) {
          bb = j;
        }
      }
      if (a < 0 || bb < 0 || __builtin_popcount(mask[a]) < 8 || __builtin_popcount(mask[bb]) < 2)
        continue;
      const uint32_t A = mask[a], B = mask[bb];
      bool ok = true;
      std::vector<int8_t> side(g.ops.size(), 0);
      // the other operands fold into B' when they fit in B (the smaller one, so the
      // fold touches fewer elements), else into A'
      for (size_t j = 0; j < g.ops.size(); ++j) {
        if ((int)j == a) side[j] = 0;
        else if ((int)j == bb) side[j] = 1;
        else if ((mask[j] & ~B) == 0u) side[j] = 1;
        else if ((mask[j] & ~A) == 0u) side[j] = 0;
        else ok = false;
      }
      const uint32_t all = g.u >= 32 ? 0xffffffffu : ((1u << g.u) - 1u);
      if (!ok || (A | B) != all) continue;
      const uint32_t Sm = (1u << g.nsum) - 1u, O = all & ~Sm;
      g.mK = Sm & A & B;
      g.mSA = Sm & A & ~B;
      g.mSB = Sm & B & ~A;
      g.mM = O & A & ~B;
      g.mN = O & B & ~A;
      g.mBt = O & A & B;
      int per_side[2] = {0, 0};
      for (int8_t sd : side) per_side[sd]++;
      if (__builtin_popcount(g.mK) > 7 || g.u > 32 || per_side[0] > 8 || per_side[1] > 8 ||
          __builtin_popcount(g.mM) > 24 || __builtin_popcount(g.mN) > 24 ||
          __builtin_popcount(g.mBt) > 24 || __builtin_popcount(g.mSA) > 8 ||
          __builtin_popcount(g.mSB) > 8)
        continue;
      g.gemm = true;
      g.gA = a;
      g.gB = bb;
      g.side = side;
    }
  }
  // triangle form of large groups with three large operands (complex64 precisions)
  if (precision != QT_FP64) {
    for (SGroup& g : S.groups) {
      if (g.u < 16 || g.ops.size() < 3 || g.nsum > 6) continue;
      std::vector<uint32_t> mask(g.ops.size(), 0u);
      for (size_t j = 0; j < g.ops.size(); ++j)
        for (int32_t l : seen_labels(g.ops[j], g.region))
          for (int b = 0; b < g.u; ++b)
            if (g.ulabels[b] == l) mask[j] |= 1u << b;
      // the three largest operands (ties: earlier operand)
      std::vector<int> idx(g.ops.size());
      for (size_t j = 0; j < idx.size(); ++j) idx[j] = (int)j;
      std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        return __builtin_popcount(mask[x]) > __builtin_popcount(mask[y]);
      });
      int a = idx[0], b = idx[1], c = idx[2];
      const uint32_t Sm = (1u << g.nsum) - 1u;
      uint32_t K = 0, X = 0, Y = 0;
      bool ok = __builtin_popcount(mask[c]) >= 4;
      for (int bit = 0; bit < g.nsum && ok; ++bit) {
        const bool ia = (mask[a] >> bit) & 1u, ib = (mask[b] >> bit) & 1u, ic = (mask[c] >> bit) & 1u;
        if (ia && ib && !ic) K |= 1u << bit;
        else if (ia && ic && !ib) X |= 1u << bit;
        else if (ib && ic && !ia) Y |= 1u << bit;
        else ok = false;  // in all three, or in one only
      }
      if (!ok) continue;
      if (__builtin_popcount(Y) > __builtin_popcount(X)) {  // Y the smaller class
        std::swap(a, b);
        std::swap(X, Y);
      }
      std::vector<int8_t> fold(g.ops.size(), 0);
      for (size_t j = 0; j < g.ops.size() && ok; ++j) {
        if ((int)j == a || (int)j == b || (int)j == c) continue;
        if ((mask[j] & ~mask[c]) == 0u) fold[j] = 1;
        else if ((mask[j] & ~K) == 0u) fold[j] = 2;
        else ok = false;
      }
      const int nx = 1 << __builtin_popcount(X), ny = 1 << __builtin_popcount(Y);
      if (!ok || ny > 4 || nx * ny > 16) continue;
      g.tri = true;
      g.tA = a;
      g.tB = b;
      g.tC = c;
      g.tK = K;
      g.tX = X;
      g.tY = Y;
      g.tfold = fold;
      g.tCbits = __builtin_popcount(mask[c]);
    }
  }
  // liveness by group: a stored tensor lives from its group to the last group reading it
  const int end_group = (int)S.groups.size();
  for (STensor& t : S.tensors) t.last_use = -1;
  for (int gi = 0; gi < end_group; ++gi)
    for (int32_t tid : S.groups[gi].ops) S.tensors[tid].last_use = gi;
  for (int32_t tid : S.scalars) S.tensors[tid].last_use = end_group;
  for (STensor& t : S.tensors)
    if (t.kind == TK_PREFIX && !t.virt && t.last_use >= 0 && t.last_use < end_group &&
        S.groups[t.last_use].region == 1)
      t.last_use = end_group;

  // memory: gates packed, prefix and slice arenas by liveness
  int64_t goff = 0;
  for (STensor& t : S.tensors)
    if (t.kind == TK_GATE) {
      t.offset = goff;
      goff += Arena::align((int64_t)1 << t.rank, kGateAlign);
    }
  S.gate_elems = goff;
  Arena pre, sl;
  for (int gi = 0; gi < end_group; ++gi) {
    SGroup& g = S.groups[gi];
    STensor& o = S.tensors[g.out];
    Arena& ar = o.kind == TK_PREFIX ? pre : sl;
    o.offset = ar.alloc((int64_t)1 << o.rank, kArenaAlign);
    if (o.last_use < 0) o.last_use = gi;
    if (g.tri) {  // C' lives only during the group
      const int64_t nc = (int64_t)1 << g.tCbits;
      g.scratch_t = ar.alloc(nc, kArenaAlign);
      ar.release(g.scratch_t, nc, kArenaAlign);
    }
    if (g.gemm) {  // A', B' live only during the group
      const int kb = __builtin_popcount(g.mK), bt = __builtin_popcount(g.mBt);
      const int64_t na = (int64_t)1 << (bt + __builtin_popcount(g.mM) + kb);
      const int64_t nb = (int64_t)1 << (bt + __builtin_popcount(g.mN) + kb);
      g.scratch_a = ar.alloc(na, kArenaAlign);
      g.scratch_b = ar.alloc(nb, kArenaAlign);
      ar.release(g.scratch_a, na, kArenaAlign);
      ar.release(g.scratch_b, nb, kArenaAlign);
    }
    for (int32_t tid : S.groups[gi].ops) {
      STensor& t = S.tensors[tid];
      if (t.kind != TK_GATE && !t.virt && t.last_use == gi)
        (t.kind == TK_PREFIX ? pre : sl).release(t.offset, (int64_t)1 << t.rank, kArenaAlign);
    }
  }
  S.prefix_elems = std::max<int64_t>(pre.top, kArenaAlign);
  S.slice_elems = std::max<int64_t>(sl.top, kArenaAlign);
  // meta slots
  int64_t shared = 0, per_slice = 0;
  for (STensor& t : S.tensors) {
    if (t.kind == TK_SLICE) t.meta = per_slice++;
    else t.meta = shared++;
  }
  S.n_shared_meta = shared;
  S.n_slice_meta_tensors = per_slice;
  for (STensor& t : S.tensors)
    if (t.kind == TK_SLICE) t.meta = shared + t.meta * S.batch;
  // workspace layout
  const size_t eb = (size_t)S.elem_bytes;
  size_t off = 0;
  // the tensor regions start on 1024 bytes, so offsets aligned to kArenaAlign elements
  // inside them are aligned in the workspace too (rows of up to 64 summed values start
  // on a whole row, as the tensor-copy GEMM kernels need)
  auto align1024 = [](size_t x) { return (x + 1023) / 1024 * 1024; };
  S.off_gates = off;
  off = align1024(off + (size_t)S.gate_elems * eb);
  S.off_prefix = off;
  off = align1024(off + (size_t)S.prefix_elems * eb);
  S.off_slices = off;
  off = align256(off + (size_t)S.slice_elems * eb * (size_t)S.batch);
  S.off_meta = off;
  off = align256(off + (size_t)(shared + per_slice * S.batch) * 16);
  S.off_partials = off;
  off = align256(off + (size_t)S.batch * (size_t)S.n_amps * 16);
  S.off_acc = off;  // n_amps accumulators, then the n_amps results
  off = align256(off + std::max<size_t>(64, (size_t)S.n_amps * 32));
  S.off_terms = off;
  off = align256(off + S.scalars.size() * kScalarTermBytes);
  S.off_segtab = off;  // step records of the segment launches (runs of small launches)
  off = align256(off + S.groups.size() * kStepRecordBytes);
  S.off_err = off;  // device status word: set when a bounded wait in a kernel gives up
  off = align256(off + 16);
  S.total_bytes = off;
  S.valid = true;
  return true;
}

std::string schedule_json(const Schedule& S, const SlicePlan& plan) {
  std::ostringstream o;
  int64_t gemm_flops = 0, tc_flops = 0, k32_flops = 0, total_flops = 0;
  int n_gemm = 0, n_tri = 0;
  for (const SGroup& g : S.groups) n_tri += g.tri;
  for (const SGroup& g : S.groups) {
    const int64_t f = g.flops * (g.region == 1 ? S.nslices : 1);
    total_flops += f;
    if (!g.gemm) continue;
    ++n_gemm;
    gemm_flops += f;
    if (__builtin_popcount(g.mM) >= 4 && __builtin_popcount(g.mN) >= 3) tc_flops += f;
    if (__builtin_popcount(g.mK) >= 5) k32_flops += f;
  }
  o << "{\"k\":" << S.k << ",\"nslices\":" << S.nslices << ",\"batch\":" << S.batch
    << ",\"n_open\":" << S.n_open
    << ",\"precision\":" << S.precision << ",\"elem_bytes\":" << S.elem_bytes
    << ",\"plan_width\":" << plan.width << ",\"slice_step\":" << plan.slice_step
    << ",\"prefix_flops\":" << S.prefix_flops << ",\"prefix_bytes\":" << S.prefix_bytes
    << ",\"slice_flops\":" << S.slice_flops << ",\"slice_bytes\":" << S.slice_bytes
    << ",\"prefix_width\":" << S.prefix_width << ",\"slice_width\":" << S.slice_width
    << ",\"n_prefix_steps\":" << S.n_prefix_steps
    << ",\"n_slice_steps\":" << (int)S.steps.size() - S.n_prefix_steps
    << ",\"n_scalars\":" << S.scalars.size() << ",\"workspace_bytes\":" << S.total_bytes
    << ",\"prefix_arena_bytes\":" << S.prefix_elems * S.elem_bytes
    << ",\"slice_arena_bytes\":" << S.slice_elems * S.elem_bytes
    << ",\"fused\":" << (S.fused ? 1 : 0) << ",\"n_groups\":" << S.groups.size()
    << ",\"gemm_groups\":" << n_gemm << ",\"tri_groups\":" << n_tri
    << ",\"job_flops\":" << total_flops
    << ",\"gemm_form_flops\":" << gemm_flops << ",\"tensor_core_shape_flops\":" << tc_flops
    << ",\"k_ge_32_flops\":" << k32_flops
    << ",\"prefix_launch_bytes\":" << S.prefix_launch_bytes
    << ",\"slice_launch_bytes\":" << S.slice_launch_bytes
    << ",\"upload_bytes\":"
    << S.gate_elems * S.elem_bytes + S.n_shared_meta * 8 +
           (int64_t)S.scalars.size() * (int64_t)kScalarTermBytes
    << ",\"steps\":[";
  for (size_t i = 0; i < S.steps.size(); ++i) {
    const SStep& st = S.steps[i];
    if (i) o << ",";
    o << "[" << st.region << "," << st.var << "," << st.ops.size() << "," << st.u << "," << st.c
      << "," << st.nsum << "," << st.flops << "," << st.bytes << "]";
  }
  o << "],\"groups\":[";
  for (size_t i = 0; i < S.groups.size(); ++i) {
    const SGroup& g = S.groups[i];
    if (i) o << ",";
    o << "[" << g.region << "," << g.first << "," << g.nsteps << "," << g.ops.size() << ","
      << g.u << "," << g.nsum << "," << g.flops << "," << g.bytes << "]";
  }
  // GEMM-form launches: first step, then the masks over the group's U bits (summed
  // in both, summed in A only, in B only, output in A only, in B only, in both) and
  // the index masks of the two large operands A and B
  o << "],\"gemm_masks\":[";
  bool first = true;
  for (const SGroup& g : S.groups) {
    if (!g.gemm) continue;
    uint32_t um[2] = {0, 0};
    for (int s = 0; s < 2; ++s) {
      const STensor& t = S.tensors[g.ops[s ? g.gB : g.gA]];
      for (int b = 0; b < g.u; ++b)
        if (std::find(t.labels.begin(), t.labels.end(), g.ulabels[b]) != t.labels.end())
          um[s] |= 1u << b;
    }
    int na = 0, nb = 0;  // operands folded into A', into B' (the large ones included)
    for (size_t j = 0; j < g.ops.size(); ++j) (g.side[j] ? nb : na)++;
    o << (first ? "" : ",") << "[" << g.first << "," << g.u << "," << g.mK << "," << g.mSA << ","
      << g.mSB << "," << g.mM << "," << g.mN << "," << g.mBt << "," << um[0] << "," << um[1]
      << "," << na << "," << nb << "]";
    first = false;
  }
  // triangle-form launches: first step, U, the summed bits of each class (K, X, Y)
  // and the index masks of the three large operands A, B, C
  o << "],\"tri_masks\":[";
  first = true;
  for (const SGroup& g : S.groups) {
    if (!g.tri) continue;
    uint32_t um[3] = {0, 0, 0};
    const int which[3] = {g.tA, g.tB, g.tC};
    for (int s = 0; s < 3; ++s) {
      const STensor& t = S.tensors[g.ops[which[s]]];
      for (int b = 0; b < g.u; ++b)
        if (std::find(t.labels.begin(), t.labels.end(), g.ulabels[b]) != t.labels.end())
          um[s] |= 1u << b;
    }
    o << (first ? "" : ",") << "[" << g.first << "," << g.u << "," << g.tK << "," << g.tX << ","
      << g.tY << "," << um[0] << "," << um[1] << "," << um[2] << "]";
    first = false;
  }
  o << "]}";
  return o.str();
}

}  // namespace qt
