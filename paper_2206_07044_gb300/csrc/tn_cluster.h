// Cluster-size choice for the one-matrix-per-cluster kernels (QR, Jacobi).
//
// A batch of B matrices, each on a cluster of P CTAs, runs in
// ceil(B / resident(P)) waves, where resident(P) is how many such clusters the
// GPU can hold at once (a cluster must fit inside one GPC, so large clusters
// can leave SMs idle).  The work of one matrix splits over its P CTAs, so the
// time goes as waves(P) / P; the chooser minimises that over a range of P.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

namespace tnk {

// Runs set(), which sets function attributes and returns a cudaError_t, once
// per (key, device): CUDA function attributes belong to the device's context,
// so a process that uses several GPUs must set them on each.  A pair is marked
// done only when set() succeeded (a failure is retried on the next launch and
// returned to the caller, who reports it as a launch error).
template <typename F>
inline cudaError_t once_per_device(const void* key, F set) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, bool> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  bool& d = done[{key, dev}];
  if (d) return cudaSuccess;
  e = set();
  if (e == cudaSuccess) d = true;
  return e;
}

// Clusters of `cluster` CTAs (threads, dynamic smem bytes) of kernel `func` that
// can be resident at once on the current device (0 if none or on error).
inline int resident_clusters(const void* func, int cluster, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int, int, size_t>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(dev, func, cluster, threads, smem);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, func, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = n;
  return n;
}

// Dynamic shared memory that leaves room for one CTA per SM at most (the
// residency query then counts clusters whose CTAs each own an SM).
inline size_t one_cta_per_sm_smem(size_t smem) {
  static std::mutex mu;
  static std::map<int, size_t> half_of;  // per device
  int dev = 0;
  cudaGetDevice(&dev);
  size_t half = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = half_of.find(dev);
    if (it != half_of.end()) half = it->second;
  }
  if (!half) {
    int per_sm = 0;
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 0;
    }
    half = (size_t)per_sm / 2 + 1024;
    std::lock_guard<std::mutex> lk(mu);
    half_of[dev] = half;
  }
  return smem > half ? smem : half;
}

// Best P in [lo, hi] for `batch` matrices; smem_of(P) gives the dynamic shared
// memory of a launch with P CTAs per cluster ((size_t)-1 to skip that P),
// imbalance(P) >= 1 the factor by which per-CTA work exceeds an even split and
// threads_of(P) the CTA size.  With one_per_sm, waves are counted for clusters
// whose CTAs each own an SM (for kernels bound by a per-SM pipe, where two CTAs
// on one SM run at half speed each).  Returns 0 when no P in the range can be
// placed.
template <typename SmemFn, typename ImbFn, typename ThrFn>
int choose_cluster(const void* func, int batch, int lo, int hi, SmemFn smem_of, ImbFn imbalance, ThrFn threads_of,
                   bool one_per_sm) {
  int best = 0;
  double best_cost = 1e300;
  for (int P = hi; P >= lo; --P) {
    const size_t smem = smem_of(P);
    if (smem == (size_t)-1) continue;
    const int threads = threads_of(P);
    int r = resident_clusters(func, P, threads, smem);
    if (one_per_sm && r > 0) {
      const int r1 = resident_clusters(func, P, threads, one_cta_per_sm_smem(smem));
      if (r1 > 0) r = r1;
    }
    if (r < 1) continue;
    const int waves = (batch + r - 1) / r;
    const double cost = (double)waves / P * imbalance(P);
    if (cost < best_cost * (1.0 - 1e-9)) {
      best_cost = cost;
      best = P;
    }
  }
  return best;
}

template <typename SmemFn, typename ImbFn>
int choose_cluster(const void* func, int threads, int batch, int lo, int hi, SmemFn smem_of, ImbFn imbalance) {
  return choose_cluster(func, batch, lo, hi, smem_of, imbalance, [threads](int) { return threads; }, false);
}

}  // namespace tnk
