// Continuous-batching request server over the C ABI.
//
// Requests (a lattice, its initial state and parameters, a step budget and an
// optional stop criterion on the change of total solid volume) queue on the
// host.  Each call to pslbm_server_advance runs one scheduling chunk:
//   1. admit queued requests in arrival order while the device-memory estimate
//      of the resident simulations stays within the HBM budget (and below the
//      resident cap);
//   2. when the resident set changed, re-pack one batch per species count (one
//      tile list and one launch per kernel for all its members), with the
//      kernel variant the first batch of that species count chose by timing;
//   3. advance every batch by `chunk_steps` steps; members whose step budget
//      ends inside the chunk are frozen on the device at their budget;
//   4. retire requests that reached their budget or whose total solid volume
//      changed by at least their stop fraction: their final budget (and, if
//      asked, their fields) is kept on the host and their device memory freed.
// Work of newly admitted requests overlaps with the running ones in the same
// batch launches; results do not depend on the mix because every simulation's
// arithmetic is per node and per instance.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/pslbm.h"

namespace {

struct Request {
  uint64_t id = 0;
  std::vector<uint8_t> mask;
  std::vector<double> rho1, rho2, conc, vol;
  pslbm_params p{};
  int64_t step_budget = 0;
  double stop_dv = 0.0;
  int keep_fields = 0;
  uint64_t bytes = 0;
  // runtime
  pslbm_t h = nullptr;
  int state = 0;  // PSLBM_REQ_*
  double v0 = 0.0;
  int64_t steps_done = 0;
  std::vector<double> budget;
  std::map<uint32_t, std::vector<unsigned char>> fields;
  std::string error;
};

}  // namespace

struct pslbm_server_s {
  pslbm_server_config cfg{};
  std::deque<Request*> queue;
  std::vector<Request*> active;
  std::map<uint64_t, std::unique_ptr<Request>> all;
  std::map<int, pslbm_batch_t> batches;   // by species count
  // the kernel variant (tile x, tile y, staging) the first batch of a species
  // count chose by timing, fixed for the batches re-packed after it
  std::map<int, std::vector<int32_t>> variant;
  bool dirty = true;
  uint64_t used = 0;
  uint64_t next_id = 1;
  double* d_budget = nullptr;             // device buffer for the allocation-free budget
  std::string err;
};

namespace {

pslbm_status sfail(pslbm_server_t s, pslbm_status st, const std::string& m) {
  if (s) s->err = m;
  return st;
}

void drop_batches(pslbm_server_t s) {
  for (auto& kv : s->batches) pslbm_batch_destroy(kv.second);
  s->batches.clear();
}

// Total solid volume and the budget of a resident simulation (no allocation).
pslbm_status read_budget(pslbm_server_t s, Request* r, std::vector<double>& out) {
  const int n = 6 + r->p.n_species;
  pslbm_status st = pslbm_budget_device_noalloc(r->h, s->d_budget);
  if (st != PSLBM_OK) return st;
  out.assign(n, 0.0);
  cudaError_t e = cudaMemcpyAsync(out.data(), s->d_budget, n * sizeof(double), cudaMemcpyDeviceToHost,
                                  (cudaStream_t)pslbm_get_stream());
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)pslbm_get_stream());
  return e == cudaSuccess ? PSLBM_OK : PSLBM_ERR_CUDA;
}

void retire(pslbm_server_t s, Request* r, const std::vector<double>& b) {
  r->budget = b;
  r->steps_done = (int64_t)b.back();
  if (r->keep_fields) {
    const size_t N = (size_t)r->p.nx * r->p.ny;
    const int ns = r->p.n_species;
    const uint32_t sel[] = {PSLBM_F_RHO1, PSLBM_F_RHO2, PSLBM_F_UX, PSLBM_F_UY, PSLBM_F_CONC, PSLBM_F_TYPE, PSLBM_F_VOL};
    const size_t sz[] = {N * 8, N * 8, N * 8, N * 8, N * ns * 8, N, 2 * N * 8};
    for (int i = 0; i < 7; ++i) {
      std::vector<unsigned char> buf(sz[i] ? sz[i] : 1);
      void* ptrs[1] = {buf.data()};
      if (sz[i] == 0) continue;
      if (pslbm_read_fields(r->h, sel[i], ptrs) == PSLBM_OK) r->fields[sel[i]] = std::move(buf);
    }
  }
  pslbm_destroy(r->h);
  r->h = nullptr;
  s->used -= r->bytes;
  r->state = PSLBM_REQ_DONE;
  r->mask.clear();
  r->mask.shrink_to_fit();
  r->rho1.clear();
  r->rho1.shrink_to_fit();
  r->rho2.clear();
  r->rho2.shrink_to_fit();
  r->conc.clear();
  r->conc.shrink_to_fit();
  r->vol.clear();
  r->vol.shrink_to_fit();
}

}  // namespace

extern "C" {

pslbm_status pslbm_server_create(const pslbm_server_config* c, pslbm_server_t* out) {
  if (!out) return PSLBM_ERR_PARAM;
  *out = nullptr;
  if (!c || c->struct_size != sizeof(pslbm_server_config)) return PSLBM_ERR_PARAM;
  if (c->chunk_steps < 1 || c->max_active < 1 || c->hbm_budget_bytes == 0 || c->precision < 0 || c->precision > 3)
    return PSLBM_ERR_PARAM;
  pslbm_server_t s = new (std::nothrow) pslbm_server_s();
  if (!s) return PSLBM_ERR_OOM;
  s->cfg = *c;
  if (cudaMalloc(&s->d_budget, (6 + PSLBM_MAX_SPECIES) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return PSLBM_ERR_NODEVICE;
  }
  *out = s;
  return PSLBM_OK;
}

pslbm_status pslbm_server_submit(pslbm_server_t s, const uint8_t* mask, const double* rho1, const double* rho2,
                                 const double* conc, const double* vol, const pslbm_params* p, int64_t step_budget,
                                 double stop_dv_frac, int32_t keep_fields, uint64_t* req_id) {
  if (!s || !mask || !rho1 || !rho2 || !p || !req_id) return sfail(s, PSLBM_ERR_PARAM, "NULL argument");
  if (step_budget < 1) return sfail(s, PSLBM_ERR_PARAM, "step budget must be >= 1");
  if (!(stop_dv_frac >= 0.0)) return sfail(s, PSLBM_ERR_PARAM, "stop fraction must be >= 0");
  pslbm_params q = *p;
  q.precision = s->cfg.precision;
  uint64_t bytes = 0;
  pslbm_status st = pslbm_estimate_device_bytes(&q, &bytes);
  if (st != PSLBM_OK) return sfail(s, st, pslbm_last_error(nullptr));
  if (bytes > s->cfg.hbm_budget_bytes) return sfail(s, PSLBM_ERR_OOM, "request alone exceeds the HBM budget");
  auto r = std::unique_ptr<Request>(new (std::nothrow) Request());
  if (!r) return PSLBM_ERR_OOM;
  const size_t N = (size_t)q.nx * q.ny;
  r->id = s->next_id++;
  r->mask.assign(mask, mask + N);
  r->rho1.assign(rho1, rho1 + N);
  r->rho2.assign(rho2, rho2 + N);
  if (conc && q.n_species) r->conc.assign(conc, conc + N * q.n_species);
  if (vol) r->vol.assign(vol, vol + 2 * N);
  r->p = q;
  r->step_budget = step_budget;
  r->stop_dv = stop_dv_frac;
  r->keep_fields = keep_fields;
  r->bytes = bytes;
  r->state = PSLBM_REQ_QUEUED;
  *req_id = r->id;
  s->queue.push_back(r.get());
  s->all[r->id] = std::move(r);
  return PSLBM_OK;
}

pslbm_status pslbm_server_advance(pslbm_server_t s, int32_t* n_active, int32_t* n_queued, int32_t* n_done) {
  if (!s) return PSLBM_ERR_PARAM;
  int32_t done_now = 0;
  // 1. admission in arrival order within the HBM budget
  while (!s->queue.empty() && (int)s->active.size() < s->cfg.max_active) {
    Request* r = s->queue.front();
    if (s->used + r->bytes > s->cfg.hbm_budget_bytes) break;
    pslbm_status st = pslbm_create(r->mask.data(), r->rho1.data(), r->rho2.data(),
                                   r->conc.empty() ? nullptr : r->conc.data(), r->vol.empty() ? nullptr : r->vol.data(),
                                   &r->p, &r->h);
    if (st == PSLBM_ERR_OOM && !s->active.empty()) break;   // wait for memory to free up
    s->queue.pop_front();
    if (st != PSLBM_OK) {
      r->state = PSLBM_REQ_FAILED;
      r->error = pslbm_last_error(nullptr);
      continue;
    }
    if ((st = pslbm_set_step_limit(r->h, r->step_budget)) != PSLBM_OK) {
      r->state = PSLBM_REQ_FAILED;
      r->error = pslbm_last_error(r->h);
      pslbm_destroy(r->h);
      r->h = nullptr;
      continue;
    }
    std::vector<double> b;
    if (read_budget(s, r, b) != PSLBM_OK) {
      // without the initial solid volume the stop criterion cannot run: the
      // request fails alone
      r->state = PSLBM_REQ_FAILED;
      r->error = std::string("initial budget read failed: ") + pslbm_last_error(r->h);
      pslbm_destroy(r->h);
      r->h = nullptr;
      continue;
    }
    r->v0 = b[3 + r->p.n_species] + b[4 + r->p.n_species];
    s->used += r->bytes;
    r->state = PSLBM_REQ_ACTIVE;
    s->active.push_back(r);
    s->dirty = true;
  }
  // 2. re-pack the batches when the resident set changed
  if (s->dirty) {
    drop_batches(s);
    std::map<int, std::vector<pslbm_t>> groups;
    for (Request* r : s->active) groups[r->p.n_species].push_back(r->h);
    for (auto& kv : groups) {
      pslbm_batch_t b = nullptr;
      auto vk = s->variant.find(kv.first);
      const bool known = vk != s->variant.end();
      pslbm_status st = pslbm_batch_create((int32_t)kv.second.size(), kv.second.data(), known ? vk->second[0] : 0,
                                           known ? vk->second[1] : 0, &b);
      if (st != PSLBM_OK) return sfail(s, st, pslbm_last_error(nullptr));
      // a staging that the new mix does not allow falls back to plain loads
      if (known && pslbm_batch_set_staging(b, vk->second[2]) != PSLBM_OK) pslbm_batch_set_staging(b, 0);
      s->batches[kv.first] = b;
    }
    s->dirty = false;
  }
  // 3. one chunk of steps for every resident simulation; the first batch of a
  // species count that a chunk tuned leaves its variant for the later ones
  for (auto& kv : s->batches) {
    pslbm_status st = pslbm_batch_step(kv.second, s->cfg.chunk_steps);
    if (st != PSLBM_OK) return sfail(s, st, pslbm_last_error(nullptr));
    if (!s->variant.count(kv.first)) {
      int32_t tx = 0, ty = 0, tuned = 0, staged = 0, avail = 0;
      if (pslbm_batch_get_tile_shape(kv.second, &tx, &ty, &tuned) == PSLBM_OK && tuned &&
          pslbm_batch_get_staging(kv.second, &staged, &avail) == PSLBM_OK)
        s->variant[kv.first] = {tx, ty, staged};
    }
  }
  if (cudaStreamSynchronize((cudaStream_t)pslbm_get_stream()) != cudaSuccess)
    return sfail(s, PSLBM_ERR_CUDA, "stream synchronisation failed");
  // 4. retire finished requests; a simulation that failed on the device
  // (non-finite density, EOS domain) is retired as failed, the others go on
  std::vector<Request*> keep;
  for (Request* r : s->active) {
    pslbm_status hs = pslbm_sync(r->h);
    if (hs == PSLBM_ERR_NONFINITE || hs == PSLBM_ERR_EOS_DOMAIN) {
      if (!s->dirty) drop_batches(s);
      s->dirty = true;
      r->error = pslbm_last_error(r->h);
      int64_t steps = 0;
      pslbm_info(r->h, &steps, nullptr, nullptr, nullptr);
      r->steps_done = steps;
      pslbm_destroy(r->h);
      r->h = nullptr;
      s->used -= r->bytes;
      r->state = PSLBM_REQ_FAILED;
      ++done_now;
      continue;
    }
    if (hs != PSLBM_OK) return sfail(s, hs, pslbm_last_error(r->h));
    std::vector<double> b;
    pslbm_status st = read_budget(s, r, b);
    if (st != PSLBM_OK) {
      // a request whose budget cannot be read fails alone; the others go on
      if (!s->dirty) drop_batches(s);
      s->dirty = true;
      r->error = std::string("budget read failed: ") + pslbm_last_error(r->h);
      pslbm_destroy(r->h);
      r->h = nullptr;
      s->used -= r->bytes;
      r->state = PSLBM_REQ_FAILED;
      ++done_now;
      continue;
    }
    r->steps_done = (int64_t)b.back();
    const double v = b[3 + r->p.n_species] + b[4 + r->p.n_species];
    const bool by_budget = r->steps_done >= r->step_budget;
    const bool by_volume = r->stop_dv > 0.0 && std::fabs(v - r->v0) >= r->stop_dv * r->v0 && r->v0 > 0.0;
    if (by_budget || by_volume) {
      if (!s->dirty) drop_batches(s);   // members leave their batch before destruction
      s->dirty = true;
      retire(s, r, b);
      ++done_now;
    } else {
      keep.push_back(r);
    }
  }
  s->active.swap(keep);
  if (n_active) *n_active = (int32_t)s->active.size();
  if (n_queued) *n_queued = (int32_t)s->queue.size();
  if (n_done) *n_done = done_now;
  return PSLBM_OK;
}

pslbm_status pslbm_server_poll(pslbm_server_t s, uint64_t id, int32_t* state, int64_t* steps_done,
                               double* budget_out) {
  if (!s) return PSLBM_ERR_PARAM;
  auto it = s->all.find(id);
  if (it == s->all.end()) return sfail(s, PSLBM_ERR_PARAM, "unknown request");
  Request* r = it->second.get();
  if (state) *state = r->state;
  if (steps_done) *steps_done = r->steps_done;
  if (budget_out && r->state == PSLBM_REQ_DONE)
    std::memcpy(budget_out, r->budget.data(), r->budget.size() * sizeof(double));
  return PSLBM_OK;
}

pslbm_status pslbm_server_fetch(pslbm_server_t s, uint64_t id, uint32_t fields, void* const* out) {
  if (!s || (fields && !out)) return PSLBM_ERR_PARAM;
  auto it = s->all.find(id);
  if (it == s->all.end()) return sfail(s, PSLBM_ERR_PARAM, "unknown request");
  Request* r = it->second.get();
  if (r->state != PSLBM_REQ_DONE || !r->keep_fields) return sfail(s, PSLBM_ERR_STATE, "no kept fields");
  int i = 0;
  for (uint32_t bit = 1; bit <= PSLBM_F_VOL; bit <<= 1) {
    if (!(fields & bit)) continue;
    auto f = r->fields.find(bit);
    if (f == r->fields.end()) return sfail(s, PSLBM_ERR_STATE, "field not kept");
    std::memcpy(out[i++], f->second.data(), f->second.size());
  }
  return PSLBM_OK;
}

pslbm_status pslbm_server_release(pslbm_server_t s, uint64_t id) {
  if (!s) return PSLBM_ERR_PARAM;
  auto it = s->all.find(id);
  if (it == s->all.end()) return sfail(s, PSLBM_ERR_PARAM, "unknown request");
  if (it->second->state == PSLBM_REQ_ACTIVE || it->second->state == PSLBM_REQ_QUEUED)
    return sfail(s, PSLBM_ERR_STATE, "request still pending");
  s->all.erase(it);
  return PSLBM_OK;
}

const char* pslbm_server_last_error(pslbm_server_t s) { return s ? s->err.c_str() : ""; }

pslbm_status pslbm_server_destroy(pslbm_server_t s) {
  if (!s) return PSLBM_OK;
  drop_batches(s);
  for (Request* r : s->active)
    if (r->h) pslbm_destroy(r->h);
  if (s->d_budget) cudaFree(s->d_budget);
  delete s;
  return PSLBM_OK;
}

}  // extern "C"
