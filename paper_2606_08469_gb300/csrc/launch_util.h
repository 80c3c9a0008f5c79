// Host helpers shared by the kernel launchers: per-kernel shared-memory
// attributes and resident CTAs per SM.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "octa_internal.h"

namespace octa {

inline int device_sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 148;
}

// Resident CTAs per SM from the kernel's registers and shared memory and the
// device limits (threads, registers, shared memory incl. the per-CTA
// reservation, CTA slots).
inline int ctas_from_resources(const void* fn, size_t smem, int threads) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) return 1;
  int dev = 0, sm_smem = 0, rsv = 0, sm_regs = 0, sm_thr = 0, sm_blk = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&sm_thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaDeviceGetAttribute(&sm_blk, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
  const int warps = (threads + 31) / 32;
  const int regs_per_warp = ((a.numRegs * 32 + 255) / 256) * 256;  // 256-register granules
  const size_t smem_cta = smem + a.sharedSizeBytes + static_cast<size_t>(rsv);
  int n = sm_blk > 0 ? sm_blk : 32;
  if (sm_thr > 0) n = std::min(n, sm_thr / (warps * 32));
  if (sm_regs > 0 && regs_per_warp > 0) n = std::min(n, sm_regs / (regs_per_warp * warps));
  if (sm_smem > 0 && smem_cta > 0) n = std::min(n, static_cast<int>(sm_smem / smem_cta));
  return std::max(1, n);
}

// Shared-memory carveout modes of the launch cache: the largest carveout
// (least L1), or the smallest one that still holds the resident CTAs (the
// rest of the SM's 256 KB of L1 / shared memory stays L1 cache).
constexpr int kCarveMaxShared = 1, kCarveFit = 2;

// Shared memory one CTA of the kernel takes (smem dynamic bytes plus its
// static and reserved bytes) and the SM's shared memory: the inputs of the
// carveout preference below.
inline void cta_shared_bytes(const void* fn, size_t smem, size_t* cta_bytes, int* sm_smem) {
  cudaFuncAttributes a;
  int dev = 0, rsv = 0;
  *sm_smem = 0;
  *cta_bytes = smem;
  if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) return;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  *cta_bytes = smem + a.sharedSizeBytes + static_cast<size_t>(rsv);
}

// The carveout preference, in percent of the SM's shared memory, that holds
// n CTAs of cta_bytes each, rounded up (the preference covers the bytes; the
// driver rounds a preference up to the next configuration it supports).
inline int fit_carveout_percent(size_t cta_bytes, int sm_smem, int n) {
  if (sm_smem <= 0) return 100;
  const size_t need = static_cast<size_t>(n) * cta_bytes;
  const size_t pct = (need * 100 + static_cast<size_t>(sm_smem) - 1) / static_cast<size_t>(sm_smem);
  return static_cast<int>(std::min<size_t>(100, pct));
}

// Sets the kernel's dynamic shared-memory limit and the largest shared-memory
// carveout, then returns the resident CTAs per SM.  For kernels that
// allocate tensor memory (tmem_cols > 0) the count comes from the kernel's
// registers and shared memory (the runtime's occupancy query reports one CTA
// per SM for them) and is capped by the 512 tensor-memory columns of an SM.
// Called once per kernel, device and shared-memory size, outside any stream
// capture; attr_smem (>= smem) is the largest size this kernel is launched
// with, which the dynamic shared-memory limit must keep allowing.
inline int resident_ctas(const void* fn, size_t smem, size_t attr_smem, int threads, int tmem_cols,
                         int* out) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(attr_smem));
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "cudaFuncSetAttribute(smem): %s", cudaGetErrorString(e));
  e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess)
    return fail(OCTA_ECUDA, "cudaFuncSetAttribute(carveout): %s", cudaGetErrorString(e));
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
  if (e != cudaSuccess) return fail(OCTA_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
  if (occ < 1) return fail(OCTA_ECUDA, "kernel does not fit on an SM (%zu B shared)", smem);
  if (tmem_cols > 0) occ = std::min(ctas_from_resources(fn, smem, threads), 512 / tmem_cols);
  *out = std::max(1, occ);
  return OCTA_OK;
}

// Cache of resident_ctas() per (kernel, device, shared-memory size), and the
// carveout each kernel was last given: get() applies the requested mode's
// carveout for that launch when it differs from the kernel's current one
// (a host-side attribute change; launches of one stream capture keep one
// mode per kernel).  cap (> 0): the launch keeps at most that many CTAs per
// SM resident, and the fitted carveout holds only those.
class LaunchCache {
 public:
  int get(const void* fn, size_t smem, int threads, int tmem_cols, int* out,
          int carve = kCarveMaxShared, int cap = 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu_);
    size_t attr = smem;
    int hit = -1;
    for (int i = 0; i < n_; ++i) {
      if (e_[i].fn != fn || e_[i].dev != dev) continue;
      if (e_[i].smem == smem) hit = i;
      attr = std::max(attr, e_[i].smem);
    }
    if (hit < 0) {
      int per_sm = 0;
      int rc = resident_ctas(fn, smem, attr, threads, tmem_cols, &per_sm);
      if (rc) return rc;
      if (n_ >= kMax) {
        *out = per_sm;
        return OCTA_OK;  // the largest carveout stays set
      }
      size_t cta_bytes = smem;
      int sm_smem = 0;
      cta_shared_bytes(fn, smem, &cta_bytes, &sm_smem);
      e_[n_] = Entry{fn, dev, smem, per_sm, cta_bytes, sm_smem};
      hit = n_++;
      set_current(fn, dev, 100);
    }
    const Entry& en = e_[hit];
    const int resident = cap > 0 ? std::min(en.per_sm, cap) : en.per_sm;
    const int want =
        carve == kCarveFit ? fit_carveout_percent(en.cta_bytes, en.sm_smem, resident) : 100;
    if (current(fn, dev) != want) {
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, want);
      if (e != cudaSuccess)
        return fail(OCTA_ECUDA, "cudaFuncSetAttribute(carveout): %s", cudaGetErrorString(e));
      set_current(fn, dev, want);
    }
    *out = e_[hit].per_sm;
    return OCTA_OK;
  }

 private:
  struct Entry {
    const void* fn;
    int dev;
    size_t smem;
    int per_sm;
    size_t cta_bytes;  // shared memory of one CTA incl. static and reserved bytes
    int sm_smem;       // the SM's shared memory (0: unknown, largest carveout)
  };
  struct Carve {
    const void* fn;
    int dev;
    int pct;
  };
  int current(const void* fn, int dev) const {
    for (int i = 0; i < nc_; ++i)
      if (c_[i].fn == fn && c_[i].dev == dev) return c_[i].pct;
    return 100;
  }
  void set_current(const void* fn, int dev, int pct) {
    for (int i = 0; i < nc_; ++i)
      if (c_[i].fn == fn && c_[i].dev == dev) {
        c_[i].pct = pct;
        return;
      }
    if (nc_ < kMax) c_[nc_++] = Carve{fn, dev, pct};
  }
  static constexpr int kMax = 256;
  Entry e_[kMax];
  int n_ = 0;
  Carve c_[kMax];
  int nc_ = 0;
  std::mutex mu_;
};

inline LaunchCache& launch_cache() {
  static LaunchCache c;
  return c;
}

// Process-wide launch knobs (octa_set_tuning); zero fields mean "default".
inline octa_tuning& tuning() {
  static octa_tuning t{};
  return t;
}
inline std::mutex& tuning_mutex() {
  static std::mutex m;
  return m;
}
inline octa_tuning tuning_snapshot() {
  std::lock_guard<std::mutex> lock(tuning_mutex());
  return tuning();
}
// The carveout mode of the launch-cache kernels (l1_carveout knob, 0 = the
// default).
constexpr int kDefaultCarve = kCarveFit;
inline int carve_mode(const octa_tuning& t) {
  return t.l1_carveout == kCarveFit || t.l1_carveout == kCarveMaxShared ? t.l1_carveout
                                                                        : kDefaultCarve;
}
// Resident CTAs per SM after an optional cap (0 = no cap).
inline int apply_cap(int per_sm, int cap) { return cap > 0 ? std::max(1, std::min(per_sm, cap)) : per_sm; }

}  // namespace octa
