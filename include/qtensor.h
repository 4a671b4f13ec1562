/*
 * qtensor.h -- C ABI of the GB300 sliced bucket-elimination QAOA simulator.
 *
 * The library computes the amplitude <z| psi_p(gamma, beta) > of the QAOA
 * MaxCut ansatz (Sec. III.A of "Tensor Network Quantum Simulator With
 * Step-Dependent Parallelization", arXiv:2012.02430) by bucket elimination of
 * its line-graph tensor network (Sec. IV, Alg. 1) under step-dependent slicing
 * (Sec. VI.C-D, Eq. 2). Every slice is an independent contraction on the GPU;
 * the slice results are summed in FP64.
 *
 * Conventions shared by every entry point:
 *   - Every call returns a qt_status and never throws or aborts. On failure the
 *     message of the calling thread's last error is available from
 *     qt_last_error(); a failed call leaves the network as it was unless its
 *     comment says otherwise.
 *   - The library copies every input array; outputs go into caller buffers.
 *   - The library allocates no device memory. Device work runs in a caller
 *     workspace (a device pointer and its size in bytes; size from
 *     qt_prepare, base aligned to 256 bytes) on the caller's CUDA stream
 *     (a cudaStream_t passed as void*, NULL for the legacy default stream).
 *   - A network is not thread-safe: calls on one qt_net must not overlap.
 *     Distinct networks are independent.
 *   - Calls that need a GPU return QT_ECUDA when the CUDA runtime reports an
 *     error; host-only calls (build, order, slice, schedule queries) need none.
 */
#ifndef QTENSOR_H
#define QTENSOR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qt_net qt_net; /* opaque, owned by the library, freed by qt_free */

typedef enum {
  QT_OK = 0,
  QT_EINVAL = 1,   /* bad argument: null pointer, out-of-range value, non-simple graph */
  QT_ENOMEM = 2,   /* host allocation failed, or the workspace is too small */
  QT_ECUDA = 3,    /* the CUDA runtime reported an error */
  QT_ETIMEOUT = 4, /* a bounded device-side wait ran out */
  QT_ESTATE = 5,   /* call made in the wrong order (e.g. contract before order) */
  QT_ERANGE = 6    /* a tensor rank exceeds what the kernels address (32) */
} qt_status;

/* Ordering rules (Sec. V.A.1). Ties always go to the smaller vertex id. */
enum {
  QT_GREEDY_MINFILL = 0, /* key (fill-in, degree, id) */
  QT_GREEDY_MINDEG = 1   /* key (degree, id): the paper's "lowest-degree vertex" */
};

/* Arithmetic of the bucket steps. Slice accumulation is FP64 in every mode. */
enum {
  QT_FP32_SIMT = 0, /* complex64 tensors, FP32 CUDA-core arithmetic */
  QT_TF32 = 1,      /* complex64; GEMM-form launches on the tensor cores in TF32 */
  QT_BF16 = 2,      /* complex64; GEMM-form launches in BF16 with FP32 accumulation */
  QT_3XTF32 = 3,    /* complex64; GEMM-form launches in split TF32 (hi*hi+hi*lo+lo*hi) */
  QT_FP64 = 4       /* complex128 tensors, FP64 CUDA-core arithmetic */
};
/* A launch is in GEMM form when its two largest tensors A, B hold every index of
 * its union and every other tensor's indices lie inside A or inside B; then it
 * is out[bt][m][n] = sum_k A'[bt][m][k] B'[bt][n][k] (k summed indices of both,
 * m/n output indices of A/B only, bt of both; A' = A times the tensors folded
 * into it, summed over indices only A sums), computed by pack kernels (planar
 * re/im) and a batched complex GEMM: on the tensor cores (mma.sync m16n8k8 TF32,
 * m16n8k16 BF16) in the TF32/BF16/3XTF32 modes when it has at least one full
 * 16 x 8 tile, else on CUDA cores in FP32. Other launches use the FP32 kernels. */

/*
 * Builds the tensor network of <z| U(gamma, beta) |+>^N (Sec. III.A; Sec. IV.A,
 * Table I; line graph with diagonal gates, Sec. IV.B, Fig. 2).
 *   edges       n_edges pairs (u, v), int32, row-major [n_edges][2]; the graph
 *               must be simple (no loops, no repeated edge), ids in [0, n_vertices)
 *   p           QAOA depth >= 1; gammas, betas: p doubles each (layer 1 first)
 *   bitstring   n_vertices bytes, each 0 or 1 (bit v is qubit v)
 *   out         receives the new network; free it with qt_free
 * Variables are (v, k), k = 0..p-1, with id k*N + v. Tensors, in order: |+> on
 * (v,0) for each v; then per layer k the phase exp(-i gamma_k [a != b]) on each
 * edge's (u,k-1),(v,k-1), then the mixer <a'|exp(-i beta_k X)|a> on
 * (v,k-1),(v,k) (k < p) or its row a' = z_v on (v,p-1) (k = p). The factor
 * 2^(-N/2) of |+>^N is applied once to the final FP64 sum.
 * Errors: QT_EINVAL for a null pointer, n_vertices < 1, p < 1, an edge id out
 * of range, a loop or repeated edge, a bit that is not 0/1, more than 2^20
 * variables; QT_ENOMEM on host allocation failure.
 */
qt_status qt_build_network(const int32_t* edges, int32_t n_vertices, int32_t n_edges, int32_t p,
                           const double* gammas, const double* betas, const uint8_t* bitstring,
                           qt_net** out);

/* Replaces the angles of a built network (order, slices and schedule are kept:
 * they depend only on the structure, Sec. VIII conclusion / Fig. 7 caption).
 * A later qt_upload is needed before device-resident runs see the new data. */
qt_status qt_set_angles(qt_net* net, const double* gammas, const double* betas);

/* Replaces the target bitstring (n_vertices bytes, 0/1); as qt_set_angles. */
qt_status qt_set_bitstring(qt_net* net, const uint8_t* bitstring);

/*
 * A batch of 2^a amplitudes in one contraction (Sec. VII): the last mixer of
 * each listed qubit keeps its output index open instead of being fixed to z_v.
 * Open qubit j (qubits[j], distinct, in [0, n_vertices)) becomes variable
 * n_vertices*p + j; the open indices form a clique of the line graph, are never
 * eliminated nor sliced, and the result is a tensor over them: entry b
 * (bit j of b = value of qubit qubits[j]) is the amplitude of the bitstring z
 * with those qubits replaced. The bits of z at open qubits are ignored.
 * a = 0 (qubits may be NULL) returns to a single amplitude. Discards the order,
 * slicing and schedule (call qt_order again). qt_run then writes 2^a
 * amplitudes; qt_contract_batch returns them.
 * Errors: QT_EINVAL for a < 0, a > QT_MAX_OPEN, a null list with a > 0, a
 * repeated or out-of-range qubit.
 */
enum { QT_MAX_OPEN = 16 };
qt_status qt_set_open(qt_net* net, const int32_t* qubits, int32_t a);

/*
 * Greedy elimination order of the line graph (Sec. V.A.1) and its contraction
 * width c = max over steps of the eliminated vertex's neighbour count
 * (Sec. IV.B). seed is reserved for randomised rules and ignored by the greedy
 * ones. Discards any earlier slicing. width_out may be NULL.
 * Errors: QT_EINVAL for an unknown algo; QT_ESTATE never (any built network).
 */
qt_status qt_order(qt_net* net, int32_t algo, uint64_t seed, int32_t* width_out);

/*
 * Randomised greedy order "rgreedy" (Sec. V.A.2): each step eliminates vertex v
 * with probability proportional to exp(-N_G(v)/tau) (N_G(v): its current
 * neighbour count); the elimination is repeated q times from one SplitMix64
 * stream seeded with `seed` (one uniform draw per step, vertices scanned in
 * ascending id; weights r^(N_G(v) - min N_G) with r = exp(-1/tau)) and the
 * order with the smallest (width, sum of 2^w, run) is kept. Open indices are
 * never taken. A later qt_slice re-orders with QT_GREEDY_MINDEG, the rule that
 * rgreedy randomises. Errors: QT_EINVAL for tau <= 0, a non-finite tau or q < 1.
 */
qt_status qt_order_rgreedy(qt_net* net, double tau, int32_t q, uint64_t seed, int32_t* width_out);

/*
 * Step-dependent slicing (Sec. VI.C-D, Fig. 8, Alg. 1). Rounds repeat while the
 * plan's width exceeds width_limit and fewer than max_vars vertices are sliced.
 * A round orders the current graph greedily (rule of qt_order), and for every
 * step s up to the first peak eliminates the first s vertices, removes the r
 * vertices with most neighbours one at a time (ties: smaller id), re-orders the
 * rest and keeps the s with the smallest (width, sum of 2^w, s).
 * Execution: steps before the first round's s run once unsliced; all k sliced
 * indices are fixed from there on, one independent contraction per slice id
 * (bit j of the id = value of the j-th sliced vertex).
 * k_out (number of sliced vertices) and width_out (plan width) may be NULL.
 * Errors: QT_ESTATE before qt_order; QT_EINVAL for width_limit < 1, r < 1,
 * max_vars < 0 or max_vars > 62 (slice ids are 64-bit; 2^k slices).
 */
qt_status qt_slice(qt_net* net, int32_t width_limit, int32_t max_vars, int32_t r, int32_t* k_out,
                   int32_t* width_out);

/* Copies of the integer plan, for bit-exact checks. Each writes at most `cap`
 * entries and stores the full length in *len. Errors: QT_ESTATE before
 * qt_order (qt_get_slices: before qt_order), QT_EINVAL for a null len. */
qt_status qt_get_order(const qt_net* net, int32_t* order, int32_t cap, int32_t* len);
qt_status qt_get_widths(const qt_net* net, int32_t* widths, int32_t cap, int32_t* len);
/* sliced vertices in slice-bit order, and the first round's step s_1 */
qt_status qt_get_slices(const qt_net* net, int32_t* vars, int32_t cap, int32_t* len,
                        int32_t* slice_step);

/*
 * Number of tensors and their labels (variable ids, in the gate's own axis
 * order) and FP64 data (interleaved re, im; axis t of the labels is bit t of
 * the element index). labels/data may be NULL to query sizes only.
 */
qt_status qt_get_tensor(const qt_net* net, int32_t t, int32_t* labels, int32_t* rank,
                        double* data);
qt_status qt_num_tensors(const qt_net* net, int32_t* count, int32_t* n_vars);

/*
 * Compiles the execution schedule for `precision` with `batch` slices per
 * device pass (batch >= 1; clamped to the number of slices) and returns the
 * workspace it needs. The schedule follows Alg. 1 with the slicing above:
 * canonical layouts (indices ordered by elimination position, earliest = least
 * significant bit; sliced indices above all others), one fused product +
 * sum-out kernel per bucket. Errors: QT_ESTATE before qt_order; QT_EINVAL for
 * an unknown precision or batch < 1; QT_ERANGE if a tensor rank exceeds 32.
 */
qt_status qt_prepare(qt_net* net, int32_t precision, int32_t batch, size_t* workspace_bytes);

/*
 * Integer ledger of the prepared schedule (per Alg. 1 step over complex
 * elements of e bytes: bytes = e (sum over operands of 2^rank + 2^c), flops =
 * 6 (m - 1) 2^u + 2 (2^u - 2^c) for m operands over union rank u), written as
 * one JSON object into buf (NUL-terminated, truncated to cap). *needed receives
 * the full length + 1. Errors: QT_ESTATE before qt_prepare.
 */
qt_status qt_stats(const qt_net* net, char* buf, size_t cap, size_t* needed);

/*
 * The prepared schedule's slice-phase launches as a captured run orders them,
 * as one JSON object into buf (as qt_stats): {"streams": S, "launches": [{"group",
 * "g_last" (the schedule groups it covers), "kind", "stream" (0 .. S-1), "wait"
 * (earlier launches on other streams it waits for), "reads", "writes" (per-slice
 * arena element ranges [lo, hi))}, ...]}. Launches on one stream run in order.
 * Two launches that write what the other reads or writes are ordered by their
 * stream or by a chain of waits. Host work only. Errors: QT_ESTATE before
 * qt_prepare; QT_ERANGE if the schedule's launches cannot be built.
 */
qt_status qt_launch_plan(qt_net* net, char* buf, size_t cap, size_t* needed);

/*
 * Copies the gate tensors (in the prepared precision and canonical layout) into
 * the workspace, asynchronously on `stream`. The host source is a staging
 * buffer owned by the network: it must not be modified (qt_set_angles) before
 * the stream has passed this copy. Errors: QT_ESTATE before qt_prepare;
 * QT_ENOMEM if workspace_bytes is below the prepared size; QT_EINVAL for a
 * workspace not aligned to 256 bytes; QT_ECUDA.
 */
qt_status qt_upload(qt_net* net, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Device-resident run: contracts slices [first, first + count) of the uploaded
 * network and writes their FP64 sum (times 2^(-N/2)) as two doubles (re, im)
 * to the DEVICE pointer d_out, asynchronously on `stream`; no host copy, no
 * synchronisation. With a open qubits (qt_set_open) d_out receives 2^a such
 * pairs, amplitude b at d_out[2b], d_out[2b+1]. The unsliced prefix (contract_first) is recomputed by every
 * call. The workspace must hold the upload of the current schedule: QT_ESTATE
 * when qt_upload has not been called on this workspace since the last
 * qt_prepare (or since qt_set_angles / qt_set_bitstring), so a stale layout is
 * never read. Errors: QT_ESTATE before qt_prepare or as above; QT_EINVAL for a
 * range outside [0, 2^k) or a null d_out; QT_ENOMEM for a small workspace;
 * QT_ECUDA.
 */
qt_status qt_run(qt_net* net, int64_t first, int64_t count, void* workspace, size_t workspace_bytes,
                 void* stream, double* d_out);

/*
 * End-to-end amplitude: prepares (if the precision differs from the prepared
 * one; batch = all slices that fit the workspace), uploads the gates, runs all
 * 2^k slices and copies the result to the HOST doubles amp_re, amp_im, then
 * synchronises `stream`. Errors: as qt_prepare, qt_upload and qt_run.
 */
qt_status qt_contract(qt_net* net, int32_t precision, void* workspace, size_t workspace_bytes,
                      void* stream, double* amp_re, double* amp_im);

/*
 * As qt_contract for a network with a >= 0 open qubits (Sec. VII): writes the
 * 2^a amplitudes to the HOST array amps (2^(a+1) doubles, amplitude b at
 * amps[2b], amps[2b+1]). qt_contract itself requires a = 0 (QT_ESTATE
 * otherwise). Errors: as qt_contract; QT_EINVAL for a null amps.
 */
qt_status qt_contract_batch(qt_net* net, int32_t precision, void* workspace,
                            size_t workspace_bytes, void* stream, double* amps);

/*
 * Angle sweep of the amplitude: n_sets >= 1 angle sets (gammas, betas: n_sets * p
 * doubles each, set s at gammas[s p .. s p + p - 1]) contracted with one order,
 * one slicing and one schedule, the reuse that makes parameter scans cheap
 * (Sec. VIII). Every set's gate tensors are built on the host and uploaded in one
 * copy; then, with no host wait in between, each set's gates are copied over the
 * workspace's gate region and all slices run (the captured graph replayed). The
 * n_sets amplitudes go to the HOST array amps (2 n_sets doubles, set s at
 * amps[2s], amps[2s+1]); `stream` is synchronised once at the end. The
 * workspace must also hold the sets' gate images: prepares (batch = all slices
 * that fit beside them) when the precision differs or they do not fit. The
 * network keeps the last set's angles. Errors: QT_EINVAL for null arguments,
 * n_sets < 1 or an angle that is not finite; QT_ESTATE before qt_order or with
 * open qubits; QT_ENOMEM when one batch and the images do not fit; as
 * qt_contract otherwise.
 */
qt_status qt_contract_sweep(qt_net* net, int32_t precision, int32_t n_sets, const double* gammas,
                            const double* betas, void* workspace, size_t workspace_bytes,
                            void* stream, double* amps);

/* Plan bookkeeping: greedy ordering runs made by the last qt_order/qt_slice/
 * qt_slice_learned and the plan's cost sum over its steps of 2^width. */
qt_status qt_plan_info(const qt_net* net, int64_t* greedy_runs, double* plan_cost);

/* ---------------------------------------------------------------------------
 * Learned proposals for the slicing search (not in the paper: the search of
 * Sec. VI.C-D re-orders the graph once per candidate step, Fig. 8). A candidate
 * is (s, v): the step s of the current greedy order (s up to its first peak)
 * and the first vertex v sliced there, v among the `topv` vertices of largest
 * degree at step s (topv = 1 is the paper's max-degree rule; further vertices
 * of a round with r > 1 are still taken by largest degree). Each candidate has
 * QT_PROPOSAL_FEATURES features read off the graph at step s with no ordering
 * run (positions, widths, degrees, fill-in and density, normalised by the
 * current width). A 2-hidden-layer ReLU MLP scores them; only the `topm`
 * best-scored candidates are ordered greedily and the best verified plan by
 * (width, sum of 2^w, s, rank) is kept, so greedy ordering decides.
 * ------------------------------------------------------------------------- */
enum { QT_PROPOSAL_FEATURES = 16 };

/* Training data from the network's first slicing round (a network ordered with
 * qt_order): every candidate's features [count][QT_PROPOSAL_FEATURES], its label
 * (the plan width after slicing it, divided by the current width) and meta
 * [count][3] = (s, v, width). Writes at most cap rows; *count gets the total.
 * Each candidate costs one greedy ordering run. */
qt_status qt_slice_dataset(const qt_net* net, int32_t topv, float* features, float* labels,
                           int32_t* meta, int32_t cap, int32_t* count);

/* Slicing with learned proposals. Per round the verified (greedily ordered)
 * candidates are: the `topm` best MLP scores (params: the MLP's parameters as
 * laid out by the qt_mlp_* calls, `hidden` units; picked steps kept apart while
 * enough candidates remain), plus `spread` candidates evenly spaced in
 * (s, rank) order. NULL params: the spread set alone (the budget the model is
 * compared with); spread >= the number of candidates verifies every candidate
 * (a full scan over (s, v); with topv = 1 this is exactly qt_slice). Sets the
 * network's plan like qt_slice. Errors as qt_slice, and QT_EINVAL for topv < 1,
 * topm < 0, spread < 0, an empty verified set, or hidden out of [1, 1024]. */
qt_status qt_slice_learned(qt_net* net, const float* params, int32_t hidden, int32_t width_limit,
                           int32_t max_vars, int32_t r, int32_t topv, int32_t topm, int32_t spread,
                           int32_t* k_out, int32_t* width_out);

/* The MLP's forward pass on the host, as qt_slice_learned uses it: x [batch][F]
 * -> y [batch]. Parameters: W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3. */
/*
 * Learned elimination steps (the next vertex to eliminate). Not in the paper, which
 * orders greedily (Sec. V.A); a model trained on the simulator's own orderings
 * proposes, greedy judges. At a step of a greedy ordering the candidates are the
 * `topc` alive vertices best by the greedy key of the network's rule (min-fill:
 * fill, degree, id; min-degree: degree, id); rank 0 is the vertex greedy takes.
 *
 * qt_order_dataset: along the network's greedy order (qt_order first), at every
 * `stride`-th step, each candidate's QT_PROPOSAL_FEATURES features (degree, fill
 * ratio, rank, fill and degree above rank 0's, neighbour degree mean/max/min, alive
 * fraction, step fraction, largest width so far, mean degree, edge density, shared
 * neighbours with rank 0, degree over the largest, 2-hop size; widths over the
 * greedy width) into features[count][F], its rollout label into labels[count]
 * (log2 of the sum of 2^w over the order: greedy up to the step, the candidate,
 * greedy after) and (step, vertex, rollout width) into meta[count][3]; at most cap
 * records written, *count gets the total (NULL arrays: count only). Errors:
 * QT_ESTATE before qt_order; QT_EINVAL for topc < 2 or stride < 1.
 *
 * qt_order_learned: orders the network by taking at every step the candidate (of
 * the top `topc`) with the lowest model score (params/hidden as qt_slice_learned);
 * with judge != 0 the plain greedy order replaces it unless the learned order's
 * (width, sum of 2^w) is smaller (*learned_kept tells which was kept). Sets the
 * network's order like qt_order (slicing and schedule discarded). Errors:
 * QT_EINVAL for a null argument, hidden outside 1..1024 or topc < 1.
 */
qt_status qt_order_dataset(const qt_net* net, int32_t topc, int32_t stride, float* features,
                           float* labels, int32_t* meta, int32_t cap, int32_t* count);
qt_status qt_order_learned(qt_net* net, const float* params, int32_t hidden, int32_t topc,
                           int32_t judge, int32_t* width_out, int32_t* learned_kept);

qt_status qt_mlp_forward_host(const float* params, int32_t n_features, int32_t hidden,
                              const float* x, int32_t batch, float* y);

/* GPU training of the MLP (mean-squared error, Adam with beta1 0.9, beta2 0.999,
 * eps 1e-8). The handle holds sizes and the Adam step count; parameters,
 * moments, activations and gradients live in a caller workspace
 * (qt_mlp_workspace_size). Device pointers: d_x [batch][F], d_t/d_y [batch],
 * d_grad [n_params], d_loss [1]. Reductions run in a fixed order (reproducible).
 * Errors: QT_EINVAL (null pointer, batch outside [1, max_batch], lr <= 0),
 * QT_ENOMEM (workspace too small), QT_ECUDA. */
typedef struct qt_mlp qt_mlp;
qt_status qt_mlp_create(int32_t n_features, int32_t hidden, int32_t max_batch, qt_mlp** out);
qt_status qt_mlp_workspace_size(const qt_mlp* mlp, size_t* bytes, int32_t* n_params);
/* host parameters in; resets the Adam moments and step (synchronises) */
qt_status qt_mlp_set_params(qt_mlp* mlp, void* workspace, size_t bytes, const float* params,
                            void* stream);
qt_status qt_mlp_get_params(const qt_mlp* mlp, void* workspace, size_t bytes, float* params,
                            void* stream);
qt_status qt_mlp_forward(qt_mlp* mlp, void* workspace, size_t bytes, const float* d_x,
                         int32_t batch, float* d_y, void* stream);
qt_status qt_mlp_gradients(qt_mlp* mlp, void* workspace, size_t bytes, const float* d_x,
                           const float* d_t, int32_t batch, float* d_grad, float* d_loss,
                           void* stream);
qt_status qt_mlp_train_step(qt_mlp* mlp, void* workspace, size_t bytes, const float* d_x,
                            const float* d_t, int32_t batch, float lr, float* d_loss,
                            void* stream);
void qt_mlp_free(qt_mlp* mlp);

/* Options of a network (qt_set_option):
 *   QT_OPT_FUSION  1 (default): consecutive bucket steps whose summed indices
 *                  die together run as one launch that sums several indices,
 *                  multiplying each step's own operands in at its level of the
 *                  nested sum (the arithmetic of Alg. 1, without storing the
 *                  intermediate results); 0: one launch per bucket (Alg. 1 as
 *                  printed). Changing it discards the prepared schedule.
 *   QT_OPT_GRAPHS  1 (default): qt_run captures its launches once per
 *                  (slice range, workspace, output) and replays the CUDA
 *                  graph; 0: direct launches.
 *   QT_OPT_GEMM    1: launches in GEMM form also use it in QT_FP32_SIMT mode
 *                  (CUDA-core GEMM: when every summed index is in both large
 *                  tensors, a shared-memory tiled kernel over the lowest U bits
 *                  after folding the small tensors into their side; else pack
 *                  kernels + GEMM); 2: the same, with the streaming kernel
 *                  (one thread per row of the large tensor, the small one
 *                  staged whole) where it applies; 0 (default): there only the
 *                  autotuner may pick them. Other values: QT_EINVAL. Discards
 *                  the prepared schedule.
 *   QT_OPT_SEGMENTS 1 (default): two or more consecutive small launches (union
 *                  of at most 12 indices) run as one segment launch, a block (or
 *                  a cluster of blocks, QT_OPT_SEG_CLUSTER) per slice stepping
 *                  through them level by level with barriers; results read only
 *                  inside the run stay in shared memory. 2..13: the
 *                  same with launches of at most that many union indices. 0: one
 *                  launch each. Values outside 0..13: QT_EINVAL. Discards the
 *                  prepared schedule.
 *   QT_OPT_TRIANGLE 1: launches in triangle form run it by default (complex64
 *                  precisions): three large tensors A, B, C with every summed
 *                  index in exactly two of them (K: A and B, X: A and C, Y: B
 *                  and C), the others inside C or summed-only inside K; then
 *                  out = sum_k w(k) sum_x A[k,x] sum_y B[k,y] C'[x,y], tiled over
 *                  the lowest U bits in shared memory. 0 (default): only the
 *                  autotuner may pick it. Discards the prepared schedule.
 *   QT_OPT_TMA     1 (default): the FP32 tiled GEMM and the triangle form
 *                  stage their operand blocks with tensor copies
 *                  (cp.async.bulk.tensor over 2-D tensor maps of the workspace,
 *                  completing on shared-memory mbarriers; bounded waits raise
 *                  QT_ETIMEOUT in qt_contract), when every block starts on a
 *                  whole row (the tiled GEMM: rows of up to 32 summed values;
 *                  rows of 64 use cp.async copies unless qt_autotune finds the
 *                  tensor copies faster for the launch); 0: cp.async copies by every thread. 2, 3, 4: as
 *                  1 with the tiled GEMM's register block fixed instead of
 *                  chosen by shared-memory wavefronts: 2 x 2 (2), 2 x 4 where
 *                  a second B-only index exists (3), 4 x 2 where a second
 *                  A-only index exists (4). Other values: QT_EINVAL.
 *   QT_OPT_CONCURRENT 1 (default): in a captured graph the slice-phase launches
 *                  that touch disjoint workspace ranges (results, operands and
 *                  scratch, compared as element ranges since the arena reuses
 *                  memory) run on up to 4 streams at once, joined by events;
 *                  0: one stream. Results are the same either way. Discards the
 *                  prepared schedule.
 *   QT_OPT_TCGEN05 In QT_TF32 and QT_3XTF32 modes, GEMM-form launches whose
 *                  shape allows it run on the tcgen05 tensor cores (operand rows
 *                  gathered by TMA tensor copies, split into TF32 planes in
 *                  shared memory, products accumulated in tensor memory; the
 *                  complex product as one real product of doubled size; rows
 *                  too long for shared memory are taken in chunks of the summed
 *                  values that accumulate in the same tensor-memory columns).
 *                  0 (default): that kernel is the launch's default and one of
 *                  the autotuner's candidates beside the FP32 kernels (which are
 *                  at least as accurate); other GEMM-form launches run the FP32
 *                  GEMM. Its tiles take as many output columns per product as
 *                  tensor memory allows (two accumulator buffers of 512 columns).
 *                  1: it is used wherever it applies, also after qt_autotune.
 *                  2: never; GEMM-form launches use the warp-level mma.sync
 *                  kernels as in QT_BF16 mode. 3: as 1, with tiles that instead
 *                  cover the longest run of lowest output indices (up to 16
 *                  batch values side by side, contiguous output runs, narrower
 *                  products). 4: as 1, with every work unit carrying at most 4
 *                  of the summed values (the chunked accumulation, which longer
 *                  rows need to fit shared memory, on every launch). Other
 *                  values: QT_EINVAL. Discards the prepared schedule.
 *   QT_OPT_SCALED  1: the tiled bucket kernel multiplies every operand by its
 *                  exact power-of-two scale 2^-s (result exponent sum of E_j + s_j)
 *                  in every slice, the path it otherwise takes only for a slice
 *                  with an extreme exponent (|s_j| > 30, or |sum s_j| > 60);
 *                  0 (default): that choice per slice. Values agree within
 *                  FP32 rounding. Discards the prepared schedule.
 *   QT_OPT_SEG_CLUSTER blocks per slice of a segment launch (a thread-block
 *                  cluster: each dependency level's work spread over its blocks,
 *                  every result written into each block's shared memory, one
 *                  cluster barrier per level). 0 (default): the largest of 8, 4,
 *                  2 whose clusters fill at most two blocks per SM, 1 when the
 *                  batch already fills the device; 1, 2, 4, 8: that size (lowered
 *                  to what the device can co-schedule). Other values: QT_EINVAL.
 *                  Results are the same bits for every size. Discards the
 *                  prepared schedule.
 * Errors: QT_EINVAL for a null network or an unknown option. */
enum { QT_OPT_FUSION = 1, QT_OPT_GRAPHS = 2, QT_OPT_GEMM = 3, QT_OPT_SEGMENTS = 4,
       QT_OPT_TRIANGLE = 5, QT_OPT_TMA = 6, QT_OPT_CONCURRENT = 7, QT_OPT_TCGEN05 = 8,
       QT_OPT_SCALED = 9, QT_OPT_SEG_CLUSTER = 10 };
qt_status qt_set_option(qt_net* net, int32_t option, int64_t value);

/*
 * Autotuner for the tile kernels. Runs the uploaded network's unsliced prefix
 * and first slice batch once (the results are those of a normal run), launching
 * every large step with each kernel variant (loads in flight per thread versus
 * resident blocks per SM) timed by CUDA events, and keeps the fastest variant
 * per step for later qt_run / qt_contract calls until the next qt_prepare.
 * Synchronises `stream`. The choice per step is written as a JSON array
 * [{"step", "variant", "ms": [per variant]}] into buf (as qt_stats; buf may be
 * NULL). Errors: QT_ESTATE before qt_prepare or without a current qt_upload
 * (as qt_run); workspace errors as qt_run;
 * QT_ECUDA.
 */
qt_status qt_autotune(qt_net* net, void* workspace, size_t workspace_bytes, void* stream, char* buf,
                      size_t cap, size_t* needed);

/*
 * Tracing. qt_profile(net, 1) makes later qt_run / qt_contract calls record a
 * CUDA event pair around every kernel launch on the caller's stream (a small
 * cost per launch); qt_profile(net, 0) stops. Either call drops the records.
 * qt_profile_read waits for the recorded events and writes a JSON array, one
 * object per launch: {"step", "kernel" (0 flat bucket, 1 tiled bucket,
 * 2 slice finalize + reduce, 3 GEMM form by pack + GEMM kernels, 4 tiled GEMM
 * form, 5 segment run, 6 triangle form, 7 streaming GEMM form), "slices",
 * "bytes", "flops" (the ledger's algorithmic counts for that launch), "ms"}
 * into buf (as qt_stats).
 * Errors: QT_EINVAL for a null network; QT_ECUDA if an event fails.
 */
qt_status qt_profile(qt_net* net, int32_t enable);
qt_status qt_profile_read(qt_net* net, char* buf, size_t cap, size_t* needed);

/*
 * qt_contract_static -- as qt_contract, with no caller workspace and no device
 * allocation. The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory (a plugin inside a host application that
 * owns the CUDA allocator, or a path that must not allocate), so they pass only
 * their inputs (the network) and outputs (amp_re, amp_im, host doubles).
 * All device scratch (gate copies, intermediate tensors, bookkeeping) lives in
 * one static device array of 64 MiB inside the library; every GPU on which the
 * library's module is loaded holds it until the process exits. The largest
 * slice batch whose schedule fits the array is used. The caller's own planning
 * state is left exactly as it was: a schedule prepared with qt_prepare, its
 * upload to the caller's workspace and its autotuned kernel choices stay valid
 * for later qt_run calls. A network whose schedule needs more than 64 MiB even
 * one slice at a time is rejected with QT_ENOMEM and a message giving both
 * sizes. It calls no cudaMalloc/cudaFree and creates no CUDA objects (tracing
 * and graph capture are skipped on this path).
 * Every call looks up the array's device address on the current device; the
 * first call on a device also loads the library's module there, so make that
 * first call before any stream capture. All calls on a device share the array,
 * which keeps the last call's contents (the call re-uploads and re-zeroes
 * everything it reads): calls that may overlap on the GPU (different streams
 * or threads) race and must be serialised by the caller.
 * The call synchronises `stream`. Errors: QT_EINVAL for a null argument;
 * QT_ESTATE before qt_order; QT_ENOMEM as above; QT_ETIMEOUT when a bounded
 * device wait gave up (as qt_contract); QT_ECUDA; others as qt_prepare.
 */
qt_status qt_contract_static(qt_net* net, int32_t precision, void* stream, double* amp_re,
                             double* amp_im);

/* ---------------------------------------------------------------------------
 * Batched energy: <C> = sum over edges of (1 - <Z_u Z_v>) / 2 for the same
 * ansatz, every edge contracted as its own lightcone tensor network: the
 * energy as a duplicated bra-ket expression (Sec. III.B) restricted to the
 * backward lightcone of Z_u Z_v (Sec. III.A). Gates kept: the layer-k cost gate
 * on (a, b) iff min(d(a), d(b)) <= p - k, the layer-k mixer on w iff
 * d(w) <= p - k, |+> on d(w) <= p, with d the distance to {u, v}; ket and bra
 * share each qubit's final index; Z = (1, -1) on the final indices of u and v.
 * Each network is ordered greedily (rule `algo`) and compiled like an
 * amplitude without slicing; all of them run in ONE persistent kernel launch
 * (replayed from a captured CUDA graph) whose blocks take networks, largest
 * first, from an atomic work counter.
 * ------------------------------------------------------------------------- */
typedef struct qt_energy qt_energy; /* opaque, owned by the library */

/* Builds and orders every edge's lightcone network. edges/angles as in
 * qt_build_network. Errors: QT_EINVAL (null pointer, n_vertices < 2, p < 1,
 * no edge, bad edge, non-finite angle, unknown algo), QT_ENOMEM. */
qt_status qt_energy_build(const int32_t* edges, int32_t n_vertices, int32_t n_edges, int32_t p,
                          const double* gammas, const double* betas, int32_t algo,
                          qt_energy** out);
/* New angles, same structure (orders kept). A later qt_energy_upload is needed. */
qt_status qt_energy_set_angles(qt_energy* e, const double* gammas, const double* betas);
/* Compiles all networks for `precision` and returns the workspace size. */
qt_status qt_energy_prepare(qt_energy* e, int32_t precision, size_t* workspace_bytes);
/* Copies gates and step tables into the workspace (async on `stream`). */
qt_status qt_energy_upload(qt_energy* e, void* workspace, size_t workspace_bytes, void* stream);
/* Device-resident run: writes <Z_u Z_v> per edge (FP64, edge order of the
 * input) to d_zz and the energy to d_energy (DEVICE pointers), async. */
qt_status qt_energy_run(qt_energy* e, void* workspace, size_t workspace_bytes, void* stream,
                        double* d_zz, double* d_energy);
/* Times block sizes 32..256 of the persistent kernel on the uploaded networks and
 * keeps the fastest (synchronises `stream`); threads_out may be NULL. */
qt_status qt_energy_autotune(qt_energy* e, void* workspace, size_t workspace_bytes, void* stream,
                             int32_t* threads_out);
/* End to end: prepare (if needed), upload, run, copy zz (host, may be NULL) and
 * the energy (host) back, synchronise `stream`. */
qt_status qt_energy_compute(qt_energy* e, int32_t precision, void* workspace,
                            size_t workspace_bytes, void* stream, double* zz_host,
                            double* energy_host);
/* One edge's network: greedy order (variable ids), variable count and width. */
qt_status qt_energy_get_order(const qt_energy* e, int32_t edge, int32_t* order, int32_t cap,
                              int32_t* len, int32_t* n_vars, int32_t* width);
/* JSON: edges, steps, widths histogram, ledger flops/bytes, launch shape. */
qt_status qt_energy_stats(const qt_energy* e, char* buf, size_t cap, size_t* needed);
/*
 * Angle sweep (toward parameter optimisation; the order and schedule depend only
 * on the structure, Sec. VIII): the energy for n_sets angle sets in one persistent
 * launch over (set, edge) work items, every lightcone network's order and schedule
 * reused. qt_energy_sweep_prepare (after qt_energy_prepare) lays out a workspace
 * for up to n_sets sets and returns its size. qt_energy_sweep takes gammas, betas
 * as HOST arrays [n_sets][p] (layer 1 first), builds each set's gate data on the
 * host (a staging buffer the handle owns: do not call again before the stream has
 * passed the copy), copies it with the network tables into the workspace and
 * launches; it writes the energies to the DEVICE array d_energy (n_sets doubles)
 * and, if d_zz is not NULL, <Z_u Z_v> to the DEVICE array d_zz [n_sets][n_edges].
 * Asynchronous on `stream`. Errors: QT_ESTATE before qt_energy_prepare;
 * QT_EINVAL for n_sets outside [1, the prepared size], a non-finite angle, a
 * null or unaligned pointer; QT_ENOMEM for a small workspace; QT_ECUDA.
 * qt_energy_sweep is qt_energy_sweep_upload (gate data and tables) followed by
 * qt_energy_sweep_run (the launch alone, repeatable on the uploaded sets).
 */
qt_status qt_energy_sweep_prepare(qt_energy* e, int32_t n_sets, size_t* workspace_bytes);
qt_status qt_energy_sweep_upload(qt_energy* e, int32_t n_sets, const double* gammas,
                                 const double* betas, void* workspace, size_t workspace_bytes,
                                 void* stream);
qt_status qt_energy_sweep_run(qt_energy* e, int32_t n_sets, void* workspace, size_t workspace_bytes,
                              void* stream, double* d_energy, double* d_zz);
qt_status qt_energy_sweep(qt_energy* e, int32_t n_sets, const double* gammas, const double* betas,
                          void* workspace, size_t workspace_bytes, void* stream, double* d_energy,
                          double* d_zz);

void qt_energy_free(qt_energy* e);

/* Frees a network (NULL is a no-op). */
void qt_free(qt_net* net);

/* Message of the calling thread's last error ("" if none). Valid until the
 * next call on that thread. */
const char* qt_last_error(void);

/* Library version string. */
const char* qt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QTENSOR_H */
