// Lookup-table evaluation of the information divergence (Sec. 4.1,
// "Function evaluations"): r_1(s) = s - 1 - ln s is tabulated on (0, 65] and
// r_f(s) = f r_1(s/f).  Table: kRfLutN entries at s_j = j h, h = 65/kRfLutN,
// linear interpolation between them; below the first entry the closed form,
// beyond 65 the tangent line at 65.  One table per device, in a __device__
// array filled by db_set_rf_eval.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace db {

__device__ float g_rf_lut[kRfLutN];

static std::atomic<int> g_rf_mode{DB_RF_LOG1P};
static std::mutex g_rf_mu;
static std::vector<const float*> g_rf_ptr;  // per device, nullptr until filled

const float* rf_lut_device() {
  if (g_rf_mode.load() != DB_RF_LUT) return nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_rf_mu);
  return dev < (int)g_rf_ptr.size() ? g_rf_ptr[dev] : nullptr;
}

int rf_mode() { return g_rf_mode.load(); }

}  // namespace db

using namespace db;

extern "C" db_status db_set_rf_eval(int mode) {
  if (mode != DB_RF_LOG1P && mode != DB_RF_LUT) return DB_ERR_ARG;
  db::bump_settings();
  if (mode == DB_RF_LUT) {
    std::vector<float> tab(kRfLutN);
    const double h = (double)kRfLutSmax / kRfLutN;
    for (int j = 1; j <= kRfLutN; ++j) {
      const double s = j * h;
      tab[j - 1] = (float)(s - 1.0 - std::log(s));
    }
    std::lock_guard<std::mutex> lk(g_rf_mu);
    int cur = 0, n = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cudaGetDeviceCount(&n) != cudaSuccess) return DB_ERR_CUDA;
    g_rf_ptr.assign(n, nullptr);
    for (int d = 0; d < n; ++d) {
      void* p = nullptr;
      if (cudaSetDevice(d) != cudaSuccess || cudaMemcpyToSymbol(g_rf_lut, tab.data(), kRfLutN * sizeof(float)) != cudaSuccess ||
          cudaGetSymbolAddress(&p, g_rf_lut) != cudaSuccess) {
        (void)cudaGetLastError();
        cudaSetDevice(cur);
        return DB_ERR_CUDA;
      }
      g_rf_ptr[d] = (const float*)p;
    }
    cudaSetDevice(cur);
  }
  g_rf_mode.store(mode);
  return DB_OK;
}
