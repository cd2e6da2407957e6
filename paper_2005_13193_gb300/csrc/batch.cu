// Many periodic fields of uneven sizes and their particle sets advanced
// together: one bin sort over the concatenated particles of all fields (global
// bin = first bin of the field + bin in the field) and one pass over the
// bricks of all fields per Heun step.  By default all steps run in one
// cooperative persistent launch (the sort's phases and the brick pass
// separated by grid-wide barriers); otherwise a launch per phase and step.
// With use_graph the solves of all fields and the steps are captured once in a
// CUDA graph and replayed.  Not part of the paper's method: a way of running
// many of its problems at once on one device.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ps_internal.cuh"

using namespace ps;

struct ps_plan {
  int nfields = 0;
  std::vector<ps_grid> grids;
  std::vector<int64_t> nps, pbase;  // pbase has nfields + 1 entries
  std::vector<int32_t> bin_base;    // nfields + 1 entries
  std::vector<BrickArgs> bricks;
  std::vector<int32_t> chunk;       // per field: 0 = bricks, else particles per bin
  int64_t np_total = 0, total_bins = 0;
  ps_dtype coef_t = PS_F32;
  int32_t brick[3] = {8, 8, 8};
  size_t smem = 0;        // brick kernel shared memory (fields share the brick shape)
  size_t args_size = 0;   // bytes of one field's brick-kernel arguments
  // workspace layout: byte offsets
  size_t off_args = 0, off_bintab = 0, off_binbase = 0, off_counts = 0, off_offsets = 0,
         off_scan = 0, off_binof = 0, off_rank = 0, off_pos = 0, off_ids = 0, off_quant = 0,
         off_sync = 0, ws_bytes = 0;
  std::vector<unsigned char> h_args;
  std::vector<BinField> h_bintab;
  // captured step sequence and what it was captured for
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<uintptr_t> key;
};

namespace {

ps_status read_tune_cache(const char* path, int32_t brick[3]) {
  if (!path || !*path) return PS_OK;
  FILE* f = fopen(path, "r");
  if (!f) return PS_OK;  // no cache yet: defaults
  char line[256];
  while (fgets(line, sizeof(line), f)) {
    int bx, by, bz;
    if (sscanf(line, "brick %d %d %d", &bx, &by, &bz) == 3) {
      brick[0] = bx;
      brick[1] = by;
      brick[2] = bz;
    }
  }
  fclose(f);
  return PS_OK;
}

void layout(ps_plan* p) {
  Carver c(nullptr);
  auto take = [&](size_t bytes) {
    c.used = align_up(c.used, 256);
    size_t o = c.used;
    c.used += bytes;
    return o;
  };
  const int64_t nf = p->nfields, np = p->np_total, nb = p->total_bins;
  p->off_args = take(nf * p->args_size);
  p->off_bintab = take(nf * sizeof(BinField));
  p->off_binbase = take((nf + 1) * sizeof(int32_t));
  p->off_counts = take((nb + 1) * sizeof(int32_t));
  p->off_offsets = take((nb + 1) * sizeof(int32_t));
  p->off_scan = take((scan_tmp_elems(nb) + 1) * sizeof(int32_t));
  p->off_binof = take(np * sizeof(int32_t));
  p->off_rank = take(np * sizeof(int32_t));
  p->off_pos = take(3 * np * sizeof(double));
  p->off_ids = take(np * sizeof(int64_t));
  p->off_sync = take(8 * sizeof(unsigned));
  size_t quant = 0;  // the largest intermediate a field's solve takes
  for (int f = 0; f < p->nfields; ++f)
    quant = std::max(quant, ps_spline_coeffs_workspace_size(&p->grids[f], 3, p->coef_t));
  p->off_quant = take(quant);
  p->ws_bytes = align_up(c.used, 256);
}

template <typename T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

}  // namespace

extern "C" ps_status ps_batch_plan(int nfields, const ps_grid* grids, const int64_t* nps,
                                   ps_dtype coef_t, const int32_t brick[3],
                                   const char* tune_cache, ps_plan** out) {
  if (!out) return fail(PS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nfields < 1 || nfields > 4096 || !grids || !nps)
    return fail(PS_ERR_INVALID_ARG, "need 1..4096 fields with grids and particle counts");
  if (coef_t != PS_F32 && coef_t != PS_BF16 && coef_t != PS_F16 && coef_t != PS_F32X4 &&
      coef_t != PS_BF16X4 && coef_t != PS_F16X4)
    return fail(PS_ERR_UNSUPPORTED, "batched runs need F32, BF16 or F16 coefficients (planar or nodes)");
  ps_plan* p = new ps_plan();
  p->nfields = nfields;
  p->coef_t = coef_t;
  if (brick)
    for (int d = 0; d < 3; ++d) p->brick[d] = brick[d];
  read_tune_cache(tune_cache, p->brick);
  p->grids.assign(grids, grids + nfields);
  p->nps.assign(nps, nps + nfields);
  p->pbase.assign(nfields + 1, 0);
  p->bin_base.assign(nfields + 1, 0);
  p->bricks.resize(nfields);
  p->chunk.assign(nfields, 0);
  int64_t bins = 0;
  for (int f = 0; f < nfields; ++f) {
    ps_status rc = validate_grid(&grids[f]);
    if (!rc) rc = make_brick_args(&grids[f], p->brick, &p->bricks[f]);
    if (!rc && nps[f] < 0) rc = fail(PS_ERR_INVALID_ARG, "field %d: negative particle count", f);
    if (rc) {
      delete p;
      return rc;
    }
    p->pbase[f + 1] = p->pbase[f] + nps[f];
    // a field so sparse that its bricks would hold fewer particles on average
    // than the staging threshold gathers from global memory anyway: bin it in
    // runs of particles, a block per run instead of a block per brick (the
    // runs cut the bricks' order into equal spans, so a run's particles are
    // neighbours and their gathers share cache lines)
    const double cells = (double)grids[f].n[0] * grids[f].n[1] * grids[f].n[2];
    const double per_brick =
        (double)nps[f] * p->brick[0] * p->brick[1] * p->brick[2] / cells;
    if (per_brick < tuning().batch_run_below) p->chunk[f] = kBatchChunk;
    bins += p->chunk[f] ? (nps[f] + kBatchChunk - 1) / kBatchChunk : p->bricks[f].nbins;
    if (bins >= ((int64_t)1 << 31)) {
      delete p;
      return fail(PS_ERR_INVALID_ARG, "too many bins in the batch");
    }
    p->bin_base[f + 1] = (int32_t)bins;
  }
  p->np_total = p->pbase[nfields];
  p->total_bins = bins;
  if (p->np_total >= ((int64_t)1 << 31)) {
    delete p;
    return fail(PS_ERR_INVALID_ARG, "too many particles in the batch");
  }
  p->args_size = staged_args_size();
  p->h_args.resize((size_t)nfields * p->args_size);
  p->h_bintab.resize(nfields);
  // the brick kernel's shared memory depends only on the brick shape
  std::vector<unsigned char> probe(p->args_size);
  size_t smem = 0;
  for (int f = 0; f < nfields; ++f) {
    size_t s = 0;
    ps_status rc = staged_fill_rk2(&grids[f], coef_t, p->brick, nullptr, nullptr, 0, nullptr,
                                   nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, nullptr,
                                   p->chunk[f] ? 1 : 0, nullptr, nullptr, 0, 0, probe.data(),
                                   &s);
    if (rc) {
      delete p;
      return rc;
    }
    smem = std::max(smem, s);
  }
  p->smem = smem;
  layout(p);
  *out = p;
  return PS_OK;
}

extern "C" size_t ps_batch_workspace_size(const ps_plan* plan) {
  return plan ? plan->ws_bytes : 0;
}

extern "C" int64_t ps_batch_num_particles(const ps_plan* plan) {
  return plan ? plan->np_total : 0;
}

extern "C" int64_t ps_batch_particle_base(const ps_plan* plan, int field) {
  if (!plan || field < 0 || field > plan->nfields) return -1;
  return plan->pbase[field];
}

namespace {

// The tables of one run (device pointers baked into the per-field arguments).
ps_status build_tables(ps_plan* p, const ps_batch_field* fields, double* pos, int64_t* ids,
                       float* vel, double dt, void* ws, int32_t* status) {
  int32_t* offsets = at<int32_t>(ws, p->off_offsets);
  double* pos_s = at<double>(ws, p->off_pos);
  int64_t* ids_s = at<int64_t>(ws, p->off_ids);
  int32_t* counts = at<int32_t>(ws, p->off_counts);
  int32_t* bin_of = at<int32_t>(ws, p->off_binof);
  for (int f = 0; f < p->nfields; ++f) {
    size_t s = 0;
    // the step kernel counts the next step's bins (global keys: the field's
    // first bin plus its bin; runs for fields binned in runs)
    const int nruns = p->chunk[f] ? p->bin_base[f + 1] - p->bin_base[f] : 0;
    ps_status rc = staged_fill_rk2(&p->grids[f], p->coef_t, p->brick, fields[f].coef,
                                   fields[f].scale, p->np_total, pos_s, pos,
                                   offsets + p->bin_base[f], vel, ids ? ids_s : nullptr, ids,
                                   dt, status, p->chunk[f] ? 1 : 0, counts + p->bin_base[f],
                                   bin_of, p->bin_base[f], nruns,
                                   p->h_args.data() + (size_t)f * p->args_size, &s);
    if (rc) return rc;
    BinField& bf = p->h_bintab[f];
    bf.g = make_grid_args(&p->grids[f]);
    bf.b = p->bricks[f];
    bf.pbase = p->pbase[f];
    bf.bin_base = p->bin_base[f];
    bf.chunk = p->chunk[f];
    bf.nruns = p->bin_base[f + 1] - p->bin_base[f];
  }
  return PS_OK;
}

ps_status upload_tables(ps_plan* p, void* ws, cudaStream_t st) {
  ps_status rc = check_cuda(cudaMemcpyAsync(at<char>(ws, p->off_args), p->h_args.data(),
                                            p->h_args.size(), cudaMemcpyHostToDevice, st),
                            "batch args upload");
  if (!rc)
    rc = check_cuda(cudaMemcpyAsync(at<char>(ws, p->off_bintab), p->h_bintab.data(),
                                    p->h_bintab.size() * sizeof(BinField),
                                    cudaMemcpyHostToDevice, st),
                    "batch bin table upload");
  if (!rc)
    rc = check_cuda(cudaMemcpyAsync(at<char>(ws, p->off_binbase), p->bin_base.data(),
                                    p->bin_base.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, st),
                    "batch bin base upload");
  // the host vectors are reused by the next run: wait for the copies
  if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "batch table upload sync");
  return rc;
}

// All nsteps Heun steps in one cooperative launch (its counters and barrier
// words cleared first, on the same stream).
ps_status enqueue_persistent(ps_plan* p, double* pos, int64_t* ids, int nsteps, void* ws,
                             int32_t* status, cudaStream_t st) {
  if (p->np_total == 0 || nsteps == 0) return PS_OK;
  ps_status rc = check_cuda(cudaMemsetAsync(at<int32_t>(ws, p->off_counts), 0,
                                            sizeof(int32_t) * (p->total_bins + 1), st),
                            "batch counts memset");
  if (!rc)
    rc = check_cuda(cudaMemsetAsync(at<unsigned>(ws, p->off_sync), 0, 8 * sizeof(unsigned), st),
                    "batch barrier memset");
  if (rc) return rc;
  return staged_batch_persistent(
      p->coef_t, at<char>(ws, p->off_args), at<int32_t>(ws, p->off_binbase),
      at<BinField>(ws, p->off_bintab), p->nfields, p->total_bins, p->np_total, nsteps, pos, ids,
      at<double>(ws, p->off_pos), ids ? at<int64_t>(ws, p->off_ids) : nullptr,
      at<int32_t>(ws, p->off_binof), at<int32_t>(ws, p->off_rank),
      at<int32_t>(ws, p->off_counts), at<int32_t>(ws, p->off_offsets),
      at<int32_t>(ws, p->off_scan), status, at<unsigned>(ws, p->off_sync), p->smem, st);
}

// One Heun step of every particle of every field: bin sort (positions and
// labels copied into bin order in the workspace), then the brick kernel,
// which writes the updated positions back in that order and counts their
// bins for the next step's sort.  The first step of a run counts from the
// positions (and clears the counters before the brick kernel); the others
// start at the scan of the counts the previous step took.
ps_status enqueue_step(ps_plan* p, double* pos, int64_t* ids, void* ws, int32_t* status,
                       bool first, cudaStream_t st) {
  if (p->np_total == 0) return PS_OK;
  int32_t* counts = at<int32_t>(ws, p->off_counts);
  ps_status rc;
  if (first) {
    rc = bin_run_batch(at<BinField>(ws, p->off_bintab), p->nfields, p->total_bins, p->np_total,
                       pos, at<int32_t>(ws, p->off_binof), at<int32_t>(ws, p->off_offsets),
                       at<double>(ws, p->off_pos), ids,
                       ids ? at<int64_t>(ws, p->off_ids) : nullptr, counts,
                       at<int32_t>(ws, p->off_rank), at<int32_t>(ws, p->off_scan), status, st);
    if (!rc)
      rc = check_cuda(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (p->total_bins + 1), st),
                      "batch counts clear");
  } else {
    rc = bin_rescan_counted(p->total_bins, p->np_total, pos, at<int32_t>(ws, p->off_binof),
                            at<int32_t>(ws, p->off_offsets), at<double>(ws, p->off_pos), ids,
                            ids ? at<int64_t>(ws, p->off_ids) : nullptr, counts,
                            at<int32_t>(ws, p->off_scan), status, st);
  }
  if (rc) return rc;
  return staged_batch_launch(p->coef_t, at<char>(ws, p->off_args),
                             at<int32_t>(ws, p->off_binbase), p->h_args.data(), p->bin_base.data(),
                             p->nfields, p->total_bins, p->smem, false, st);
}

}  // namespace

extern "C" ps_status ps_batch_run(ps_plan* p, const ps_batch_field* fields, int solve,
                                  double* pos, int64_t* ids, float* vel_out, int nsteps,
                                  double dt, int use_graph, void* ws, size_t ws_bytes,
                                  int32_t* status, void* stream) {
  if (!p || !fields) return fail(PS_ERR_INVALID_ARG, "plan and fields are required");
  if (nsteps < 0 || !std::isfinite(dt)) return fail(PS_ERR_INVALID_ARG, "bad nsteps or dt");
  if (p->np_total > 0 && !pos) return fail(PS_ERR_INVALID_ARG, "pos is NULL");
  if (!ws || ws_bytes < p->ws_bytes || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(PS_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", p->ws_bytes);
  const bool quant = p->coef_t == PS_BF16 || p->coef_t == PS_F16 || p->coef_t == PS_BF16X4 ||
                     p->coef_t == PS_F16X4;
  for (int f = 0; f < p->nfields; ++f) {
    if (!fields[f].coef) return fail(PS_ERR_INVALID_ARG, "field %d: coef is NULL", f);
    if (quant && !fields[f].scale) return fail(PS_ERR_INVALID_ARG, "field %d: scale is NULL", f);
    if (solve && !fields[f].field) return fail(PS_ERR_INVALID_ARG, "field %d: field is NULL", f);
  }
  cudaStream_t st = as_stream(stream);
  ps_status rc;
  const bool persistent = tuning().batch_persistent != 0;
  // the solves of all fields (into the workspace's quantisation area when the
  // storage needs an intermediate)
  auto enqueue_solves = [&](cudaStream_t s) -> ps_status {
    const size_t qbytes = p->ws_bytes - p->off_quant;
    for (int f = 0; f < p->nfields; ++f) {
      const bool inter = ps_spline_coeffs_workspace_size(&p->grids[f], 3, p->coef_t) > 0;
      ps_status r = ps_spline_coeffs(&p->grids[f], 3, PS_F32, fields[f].field, p->coef_t,
                                     fields[f].coef, fields[f].scale,
                                     inter ? at<char>(ws, p->off_quant) : nullptr,
                                     inter ? qbytes : 0, s);
      if (r) return r;
    }
    return PS_OK;
  };
  auto enqueue_steps = [&](cudaStream_t s) -> ps_status {
    if (persistent) return enqueue_persistent(p, pos, ids, nsteps, ws, status, s);
    for (int k = 0; k < nsteps; ++k) {
      ps_status r = enqueue_step(p, pos, ids, ws, status, k == 0, s);
      if (r) return r;
    }
    return PS_OK;
  };
  const bool steps = nsteps > 0 && p->np_total > 0;
  if (!use_graph) {
    if (solve && (rc = enqueue_solves(st))) return rc;
    if (!steps) return PS_OK;
    if ((rc = build_tables(p, fields, pos, ids, vel_out, dt, ws, status))) return rc;
    if ((rc = upload_tables(p, ws, st))) return rc;
    return enqueue_steps(st);
  }
  if (!solve && !steps) return PS_OK;

  std::vector<uintptr_t> key = {(uintptr_t)pos, (uintptr_t)ids, (uintptr_t)vel_out,
                                (uintptr_t)ws, (uintptr_t)status, (uintptr_t)nsteps,
                                (uintptr_t)(solve ? 1 : 0), (uintptr_t)(persistent ? 1 : 0)};
  uint64_t dtbits;
  memcpy(&dtbits, &dt, sizeof(dt));
  key.push_back((uintptr_t)dtbits);
  for (int f = 0; f < p->nfields; ++f) {
    key.push_back((uintptr_t)fields[f].coef);
    key.push_back((uintptr_t)fields[f].scale);
    key.push_back((uintptr_t)(solve ? fields[f].field : nullptr));
  }
  if (p->exec && key == p->key) return check_cuda(cudaGraphLaunch(p->exec, st), "graph launch");
  if (steps) {
    if ((rc = build_tables(p, fields, pos, ids, vel_out, dt, ws, status))) return rc;
    if ((rc = upload_tables(p, ws, st))) return rc;
  }
  if (p->exec) {
    cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
  }
  if (!p->cap &&
      (rc = check_cuda(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking),
                       "capture stream")))
    return rc;
  if ((rc = staged_batch_launch(p->coef_t, nullptr, nullptr, nullptr, nullptr, 0, 0, p->smem, true,
                                p->cap)))
    return rc;
  if ((rc = check_cuda(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal),
                       "begin capture")))
    return rc;
  ps_status cap_rc = solve ? enqueue_solves(p->cap) : PS_OK;
  if (!cap_rc && steps) cap_rc = enqueue_steps(p->cap);
  cudaGraph_t graph = nullptr;
  rc = check_cuda(cudaStreamEndCapture(p->cap, &graph), "end capture");
  if (cap_rc || rc) {
    if (graph) cudaGraphDestroy(graph);
    return cap_rc ? cap_rc : rc;
  }
  rc = check_cuda(cudaGraphInstantiate(&p->exec, graph, 0), "graph instantiate");
  cudaGraphDestroy(graph);
  if (rc) return rc;
  p->key = key;
  return check_cuda(cudaGraphLaunch(p->exec, st), "graph launch");
}

extern "C" void ps_plan_destroy(ps_plan* plan) {
  if (!plan) return;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->cap) cudaStreamDestroy(plan->cap);
  delete plan;
}
