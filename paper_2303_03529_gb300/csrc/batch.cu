// Batched replicas: many independent systems (different sizes) stepped
// together.  Each replica is an ordinary context on its own non-blocking
// stream; a pool of host threads drives them, largest first, so the small
// products of different replicas run on the GPU at the same time.  Replicas
// share nothing but the device, so a batched step gives the same result, bit
// for bit, as stepping the replica alone.
#include "common.cuh"

#include <algorithm>
#include <array>
#include <thread>

struct sxl_batch {
  std::vector<sxl_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  std::vector<int> order;  // replica indices, largest first
};

extern "C" {

int sxl_batch_create(const sxl_params* params, int count, sxl_batch** out) {
  if (!params || count < 1 || !out) return SXL_E_ARG;
  *out = nullptr;
  sxl_batch* b = new sxl_batch();
  for (int i = 0; i < count; ++i) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      sxl_batch_destroy(b);
      return SXL_E_CUDA;
    }
    b->streams.push_back(s);
    sxl_ctx* c = nullptr;
    int r = sxl_create(&params[i], (void*)s, &c);
    if (r != SXL_OK) {
      sxl_batch_destroy(b);
      return r;
    }
    b->ctx.push_back(c);
    b->order.push_back(i);
  }
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int x, int y) { return params[x].n_atoms > params[y].n_atoms; });
  *out = b;
  return SXL_OK;
}

int sxl_batch_context(sxl_batch* b, int i, sxl_ctx** out) {
  if (!b || !out || i < 0 || i >= (int)b->ctx.size()) return SXL_E_ARG;
  *out = b->ctx[i];
  return SXL_OK;
}

int sxl_batch_step(sxl_batch* b, int nsteps, int nthreads, int* status) {
  if (!b || nsteps < 0) return SXL_E_ARG;
  const int count = (int)b->ctx.size();
  if (nthreads <= 0) nthreads = std::min(count, 16);
  nthreads = std::min(nthreads, count);
  std::vector<int> rc(count, SXL_OK);
  std::atomic<int> next{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SXL_E_CUDA;
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= count) break;
      const int i = b->order[k];
      rc[i] = xlbomd_step(b->ctx[i], nsteps, nullptr);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t) pool.emplace_back(worker);
  for (std::thread& t : pool) t.join();
  int first = SXL_OK;
  for (int i = 0; i < count; ++i) {
    if (status) status[i] = rc[i];
    if (first == SXL_OK && rc[i] != SXL_OK) first = rc[i];
  }
  return first;
}

// Tile autotuning of a batch: replicas with the same chain dimension share
// one tuning run (the first of them is timed, the others take its choice).
int sxl_batch_autotune(sxl_batch* b, double* report_host) {
  if (!b) return SXL_E_ARG;
  std::vector<std::pair<int, std::array<int, 6>>> done;  // (Np, choice)
  int k = 0;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    sxl_ctx* c = b->ctx[i];
    bool found = false;
    for (auto& d : done)
      if (d.first == c->Np) {
        SXL_TRY(sxl_set_tiles(c, d.second[0], d.second[1], d.second[2], d.second[3]));
        c->tc_ps_plain = d.second[4];
        c->tc_ps_dual = d.second[5];
        found = true;
        break;
      }
    if (found) continue;
    double out[9];
    SXL_TRY(sxl_autotune(c, out));
    done.push_back({c->Np, {(int)out[0], (int)out[1], (int)out[3], (int)out[5],
                            c->tc_ps_plain, c->tc_ps_dual}});
    if (report_host) {
      double* r = report_host + 10 * k;
      r[0] = c->Np;
      for (int j = 0; j < 9; ++j) r[1 + j] = out[j];
    }
    ++k;
  }
  return k;  // distinct chain dimensions tuned
}

int sxl_batch_destroy(sxl_batch* b) {
  if (!b) return SXL_OK;
  for (sxl_ctx* c : b->ctx) sxl_destroy(c);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  delete b;
  return SXL_OK;
}

}  // extern "C"
