// Error reporting, device-pointer checks, the library's memory pools and
// grow-only device buffers.
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>

#include "pc_internal.cuh"

namespace pc {

static thread_local char g_last_error[1024] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return code;
}

void clear_error() { g_last_error[0] = 0; }

bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error state of this query
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------- memory pools

namespace {
std::mutex g_mem_mutex;
std::map<int, cudaMemPool_t> g_pools;
std::vector<std::pair<size_t, void*>> g_pinned;       // free pinned host blocks
std::map<void*, size_t> g_pinned_size;                // size of every pinned block handed out
std::map<int, std::vector<cudaStream_t>> g_streams;   // free non-blocking streams per device

cudaMemPool_t pool_of_current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mem_mutex);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) return it->second;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  uint64_t keep = ~0ull;   // keep freed memory for reuse (pc_trim_memory returns it)
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  g_pools[dev] = pool;
  return pool;
}
}  // namespace

int dmalloc(void** ptr, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 256;
  cudaMemPool_t pool = pool_of_current_device();
  if (!pool) return fail(PC_ERR_CUDA, "device memory pool could not be created");
  const cudaError_t e = cudaMallocFromPoolAsync(ptr, bytes, pool, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA,
                "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  return PC_OK;
}

void dfree(void* ptr, cudaStream_t st) {
  if (ptr) cudaFreeAsync(ptr, st);
}

void dfree_idle(void* ptr) {
  if (!ptr) return;
  cudaDeviceSynchronize();
  cudaFreeAsync(ptr, 0);
}

void* pinned_get(size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(g_mem_mutex);
    long best = -1;   // the smallest free block that fits
    for (size_t i = 0; i < g_pinned.size(); ++i)
      if (g_pinned[i].first >= bytes && (best < 0 || g_pinned[i].first < g_pinned[(size_t)best].first))
        best = (long)i;
    if (best >= 0) {
      void* q = g_pinned[(size_t)best].second;
      g_pinned.erase(g_pinned.begin() + best);
      return q;
    }
  }
  void* q = nullptr;
  const size_t want = bytes < 4096 ? 4096 : bytes;
  if (cudaMallocHost(&q, want) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mem_mutex);
  g_pinned_size[q] = want;
  return q;
}

void pinned_put(void* q) {
  if (!q) return;
  std::lock_guard<std::mutex> lk(g_mem_mutex);
  g_pinned.emplace_back(g_pinned_size[q], q);
}

cudaStream_t stream_get() {
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(g_mem_mutex);
    auto& v = g_streams[dev];
    if (!v.empty()) {
      cudaStream_t s = v.back();
      v.pop_back();
      return s;
    }
  }
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return s;
}

void stream_put(cudaStream_t s) {
  if (!s) return;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mem_mutex);
  g_streams[dev].push_back(s);
}

int trim_memory() {
  if (cudaDeviceSynchronize() != cudaSuccess)
    return fail(PC_ERR_CUDA, "pc_trim_memory: %s", cudaGetErrorString(cudaGetLastError()));
  std::lock_guard<std::mutex> lk(g_mem_mutex);
  for (auto& kv : g_pools) cudaMemPoolTrimTo(kv.second, 0);
  for (auto& b : g_pinned) {
    g_pinned_size.erase(b.second);
    cudaFreeHost(b.second);
  }
  g_pinned.clear();
  return PC_OK;
}

int DevBuf::ensure(size_t nbytes) {
  if (nbytes <= bytes && p != nullptr) return PC_OK;
  dfree_idle(p);
  p = nullptr;
  bytes = 0;
  size_t want = nbytes < 256 ? 256 : nbytes;
  PC_TRY(dmalloc(&p, want, 0));
  PC_CUDA(cudaStreamSynchronize(0));   // usable from every stream
  bytes = want;
  return PC_OK;
}

void DevBuf::release() {
  dfree_idle(p);
  p = nullptr;
  bytes = 0;
}

}  // namespace pc

extern "C" const char* pc_last_error(void) { return pc::g_last_error; }

extern "C" int pc_abi_version(void) { return PC_ABI_VERSION; }

extern "C" int pc_trim_memory(void) {
  pc::clear_error();
  return pc::trim_memory();
}

// ------------------------------------------------------------------ kernel timing

namespace pc {
namespace {

const char* const kProfNames[PROF_NCLASSES] = {"plan",     "grid",     "fft_rows", "fft_cols",
                                               "residual", "gram_fp32", "gram_finalize",
                                               "apgd",     "select",   "misc",     "gram_tc",
                                               "gram_thin", "dict_corr", "dict_columns", "phase_gen",
                                               "apgd_op", "degrid", "degrid_fft"};

struct ProfRec {
  int cls;
  int kernels;
  cudaEvent_t a, b;
};

bool g_prof_on = false;
unsigned g_prof_mask = ~0u;   // classes recorded while profiling is on
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_pool;
size_t g_pool_used = 0;

cudaEvent_t pool_event() {
  if (g_pool_used < g_pool.size()) return g_pool[g_pool_used++];
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  g_pool.push_back(e);
  ++g_pool_used;
  return e;
}

}  // namespace

bool prof_active() { return g_prof_on; }

int prof_start(int cls, cudaStream_t st) {
  if (!g_prof_on || !((g_prof_mask >> cls) & 1u)) return -1;
  cudaEvent_t a = pool_event(), b = pool_event();
  if (!a || !b) return -1;
  cudaEventRecord(a, st);
  g_prof.push_back(ProfRec{cls, 0, a, b});
  return (int)g_prof.size() - 1;
}

void prof_stop(int token, cudaStream_t st, int kernels) {
  if (token < 0 || token >= (int)g_prof.size()) return;
  cudaEventRecord(g_prof[token].b, st);
  g_prof[token].kernels = kernels;
}

}  // namespace pc

extern "C" int pc_profile_begin(void) {
  pc::g_prof.clear();
  pc::g_pool_used = 0;
  pc::g_prof_mask = ~0u;
  pc::g_prof_on = true;
  return PC_OK;
}

extern "C" int pc_profile_begin_classes(const char* classes) {
  using namespace pc;
  unsigned mask = 0;
  if (!classes || !*classes) {
    mask = ~0u;
  } else {
    std::string s(classes);
    size_t pos = 0;
    while (pos <= s.size()) {
      size_t q = s.find(',', pos);
      if (q == std::string::npos) q = s.size();
      const std::string name = s.substr(pos, q - pos);
      bool found = false;
      for (int c = 0; c < PROF_NCLASSES; ++c)
        if (name == kProfNames[c]) {
          mask |= 1u << c;
          found = true;
        }
      if (!found) return fail(PC_ERR_INVALID_ARG, "pc_profile_begin_classes: unknown class '%s'", name.c_str());
      pos = q + 1;
    }
  }
  g_prof.clear();
  g_pool_used = 0;
  g_prof_mask = mask;
  g_prof_on = true;
  return PC_OK;
}

extern "C" int pc_profile_end(pc_kernel_time* out, int32_t cap, int32_t* n_out) {
  using namespace pc;
  g_prof_on = false;
  double tot[PROF_NCLASSES] = {0};
  int64_t cnt[PROF_NCLASSES] = {0};
  int64_t nk[PROF_NCLASSES] = {0};
  for (const ProfRec& r : g_prof) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) {
      cudaGetLastError();
      return fail(PC_ERR_CUDA, "pc_profile_end: event synchronisation failed");
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      tot[r.cls] += ms;
      cnt[r.cls] += 1;
      nk[r.cls] += r.kernels;
    } else {
      cudaGetLastError();
    }
  }
  g_prof.clear();
  g_pool_used = 0;
  int n = 0;
  for (int c = 0; c < PROF_NCLASSES; ++c) {
    if (!cnt[c]) continue;
    if (out && n < cap) {
      std::snprintf(out[n].name, sizeof(out[n].name), "%s", kProfNames[c]);
      out[n].launches = cnt[c];
      out[n].kernels = nk[c];
      out[n].total_ms = tot[c];
    }
    ++n;
  }
  if (n_out) *n_out = n;
  return PC_OK;
}
