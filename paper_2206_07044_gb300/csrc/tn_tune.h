// Autotuned launch shapes: a per-device table of measured choices that the
// kernel launchers consult before their built-in rules.
//
// A key is (kernel family, m, n, k, batch) -- the shape of one launch of a
// step of the schedule -- and the value is the family's launch parameter:
//   TK_QR        cluster size P of qr_cluster_kernel
//   TK_JAC64     cluster size P of the FP64 polish (block_jacobi_kernel<double>)
//   TK_JAC32     cluster size P of the FP32 pass (block_jacobi_kernel<float>)
//   TK_GEMM64    tile variant of gemm_f64_kernel (1: 64x64, 2: 32x32, 3: 128x32, 4: 128x16)
//   TK_GEMMTC    N tile (BN) of the tcgen05 GEMM (64, 128 or 256)
// tn_autotune fills the table by timing every candidate on scratch data of
// each shape; a missing key means "use the built-in rule".  The table can be
// written to and read from a text cache file, tagged with the device name and
// SM count so that a cache taken on another GPU model is not applied.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace tnk {

enum TuneKernel : int { TK_QR = 1, TK_JAC64 = 2, TK_JAC32 = 3, TK_GEMM64 = 4, TK_GEMMTC = 5 };

// Measured choice for this key on the current device, or 0.
int tune_get(int kernel, int m, int n, int k, int batch);
// Record a choice for this key on the current device (value 0 erases it).
void tune_set(int kernel, int m, int n, int k, int batch, int value);
// Number of entries for the current device.
int tune_count();
// Every entry of the current device as (kernel, m, n, k, batch, value) rows.
std::vector<std::vector<int>> tune_entries();
// Write / read the current device's entries (text; "" on success, else an error).
std::string tune_save(const std::string& path);
std::string tune_load(const std::string& path);

}  // namespace tnk
