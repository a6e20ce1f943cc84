// Host-side declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "cox.h"
#include "cox_internal.h"

namespace coxgb {

void set_allocator(cox_alloc_fn a, cox_free_fn f, void *ctx);
void *dev_alloc(size_t bytes);
void dev_free(void *p, size_t bytes);
bool pointer_on_device(const void *p);
int64_t launch_count();
// Process-wide limit of the device-side waits (0: the default); read by every launcher.
void set_wait_limit(long long clocks);
// Record `msg` as the calling thread's last error and return `code` (api.cu).
int set_last_error(int code, const char *msg);

// Owns device buffers; releases them on destruction. Requests up to kSlabMax bytes are carved
// from slabs of kSlabBytes (one allocator call for many small tables); larger ones are
// allocations of their own. bytes_total counts the bytes handed out.
struct BufferSet {
  static constexpr size_t kSlabBytes = size_t(1) << 20, kSlabMax = size_t(1) << 16;
  std::vector<std::pair<void *, size_t>> bufs;   // the device allocations owned
  size_t bytes_total = 0;
  char *slab = nullptr;    // the current slab's unused tail
  size_t slab_left = 0;
  BufferSet() = default;
  BufferSet(const BufferSet &) = delete;
  BufferSet &operator=(const BufferSet &) = delete;
  ~BufferSet() { release(); }
  void *get(size_t bytes);
  void release();
};
using Scratch = BufferSet;

// A prepared data set: device descriptor plus the host copies the launcher needs.
struct Prepared {
  BufferSet bufs;
  DevData desc{};
  int64_t nnz_rows = 0;
  std::vector<int64_t> h_col_ptr_rows;  // row-space CSC pointers
  std::vector<int64_t> h_col_ptr;       // position-space CSC pointers
  std::vector<int32_t> h_tile_lo;       // streaming plan: first position of each tile
  std::vector<int32_t> h_tile_g;        // streaming plan: first tie group of each tile
  int32_t *strata_start = nullptr;      // [K+1] device
  // resident plan (one tile per CTA of the resident kernel); res_T == 0 when not eligible
  int32_t res_T = 0;
  int32_t *res_tile_lo = nullptr, *res_tile_g = nullptr, *res_tile_k = nullptr, *res_col_tile = nullptr;
  // incremental plan (one tile per CTA of the incremental kernel); inc_T == 0 when not eligible
  int32_t inc_T = 0;
  int32_t *inc_tile_lo = nullptr, *inc_tile_g = nullptr, *inc_tile_k = nullptr, *inc_col_tile = nullptr;
  int32_t inc_wmin = 0x7fffffff;        // shortest run of positions overflowing a column's list
  // columns too dense for the incremental lists: fits step them with the resident kernel
  int32_t inc_n_halt = 0;
  int32_t inc_variant = 0;              // kernel configuration of the plan (see inc_group_cap)
  uint8_t *inc_halt = nullptr;          // [p] device, null when none
  std::vector<uint8_t> h_inc_halt;      // [p] host copy
  // compact incremental plan (fewest tiles; batches), built on first use: 0 = not yet, -1 = none
  int32_t cinc_T = 0;
  int32_t *cinc_tile_lo = nullptr, *cinc_tile_g = nullptr, *cinc_tile_k = nullptr, *cinc_col_tile = nullptr;
  int32_t *g_time = nullptr;            // [G] device
  int32_t *g_stratum = nullptr;         // [G] device
};

int prepare_data(const cox_data *in, int precision, int tile_req, cudaStream_t s, Prepared *out, std::string *err);
// Time-split view of a data set (§2.2, §2.3), built by device kernels; its arrays are owned
// by `B` (device memory) and described by *view.
int split_columns(int32_t p, const cox_split *sp, int32_t *p_view, std::string *err);
int build_split_view(const cox_data *in, const cox_split *sp, cudaStream_t s, BufferSet &B, cox_data *view,
                     std::string *err);
// The rows whose fold id differs from k (a cross-validation training set), built on the device;
// arrays owned by `B`. Fold ids outside [0, K) are an error.
int build_fold_view(const cox_data *in, const int32_t *fold, int32_t k, int32_t K, cudaStream_t s, BufferSet &B,
                    cox_data *view, std::string *err);
// Build (once) the incremental kernel's compact plan of a prepared data set (fewest tiles).
int prepare_compact_incr(Prepared *P, int precision, cudaStream_t s, std::string *err);

}  // namespace coxgb
