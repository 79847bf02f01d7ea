// sigma_noalloc: sigma whose scratch lives in a file-scope device array, for
// callers that must not allocate device memory while they run.
#include "pno.cuh"
#include <functional>
#include <mutex>

namespace pnoeom {
int guard_call(const std::function<void()>& f);
}

namespace {

// Scratch of every sigma_noalloc call (all calls share it; see the header).
static __device__ __align__(256) unsigned char g_noalloc_scratch[PNOEOM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on `device` (which must be current).
// In host code the array's name is only a host-side stand-in, so the address
// is looked up once per device with cudaGetSymbolAddress.
void* scratch_address(int device) {
  PN_CHECK(device >= 0 && device < kMaxDevices, PNOEOM_ERR_UNSUPPORTED, "device index too large for sigma_noalloc");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    PN_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    PN_CHECK(p != nullptr, PNOEOM_ERR_CUDA, "cudaGetSymbolAddress returned NULL");
    g_scratch_addr[device] = p;
  }
  return g_scratch_addr[device];
}

template <typename T>
void sigma_into_scratch(const pnoeom_pno* P, int nvec, const T* r, T* out, T* work, cudaStream_t s, bool bf16) {
  using namespace pnoeom;
  SysTable t{};
  t.nsys = 1;
  t.max_nvec = nvec;
  t.s[0] = sysbuf(P, nvec, r, out, work, sizeof(T) == 4, bf16);
  const int64_t ol = P->L, wl = P->work_len;
  run_program<T>(P->prog, t, &ol, &wl, s, nullptr);
}

}  // namespace

extern "C" int sigma_noalloc(pnoeom_ctx* ctx, const pnoeom_pno* pno, int nvec, const void* r_dev, void* s_dev,
                             int precision, void* cuda_stream) {
  return pnoeom::guard_call([&] {
    PN_CHECK(ctx && pno, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    PN_CHECK(nvec >= 0, PNOEOM_ERR_INVALID_ARG, "nvec < 0");
    if (nvec == 0) return;
    PN_CHECK(r_dev && s_dev, PNOEOM_ERR_INVALID_ARG, "NULL vector");
    PN_CHECK(precision == PNOEOM_FP64 || precision == PNOEOM_FP32 || precision == PNOEOM_BF16, PNOEOM_ERR_INVALID_ARG,
             "unknown precision");
    const size_t elem = precision == PNOEOM_FP64 ? 8 : 4;
    const size_t need = (size_t)nvec * (size_t)pno->work_len * elem;
    PN_CHECK(need <= PNOEOM_NOALLOC_SCRATCH_BYTES, PNOEOM_ERR_UNSUPPORTED,
             "sigma_noalloc needs " + std::to_string(need) + " bytes of scratch for " + std::to_string(nvec) +
                 " vectors, more than its fixed " + std::to_string((size_t)PNOEOM_NOALLOC_SCRATCH_BYTES) +
                 "-byte array; pass fewer vectors per call or use sigma()");
    pnoeom::DeviceScope dev_scope(ctx->device);
    void* work = scratch_address(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    if (precision == PNOEOM_FP64)
      sigma_into_scratch<double>(pno, nvec, (const double*)r_dev, (double*)s_dev, (double*)work, s, false);
    else
      sigma_into_scratch<float>(pno, nvec, (const float*)r_dev, (float*)s_dev, (float*)work, s, precision == PNOEOM_BF16);
  });
}
