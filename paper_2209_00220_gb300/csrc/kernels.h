// Launchers of the sm_103a kernels (scan.cu, lookup.cu) and the device status
// word. Internal to libbytestore.
#pragma once

#include <cuda_runtime.h>

#include "bs_internal.h"

namespace bs {

// Device status bits (atomicOr'ed by kernels, read by bs_last_device_error).
constexpr uint32_t kStatusBounds = 1u;   // an index failed its bounds check
constexpr uint32_t kStatusTimeout = 2u;  // a bounded wait gave up

// status: device word the kernels report bounds / timeout flags into (NULL:
// the library's status word of the current device).
int launch_scan(const Column &c, const KPred &p, const uint32_t *d_seed, uint32_t *d_out, cudaStream_t s,
                uint32_t *status = nullptr);

uint64_t lookup_workspace_bytes(const Column &c);
// Either d_vals or d_codes is non-null.
int launch_lookup(const Column &c, const uint32_t *d_bits, int32_t *d_vals, uint64_t *d_codes, uint64_t out_cap,
                  uint64_t *d_count, void *d_ws, cudaStream_t s, uint32_t *status = nullptr);
// Launch shape bs_lookup's gather kernel takes for this column (values, not
// codes): warps per 16-tile chunk, grid, resident CTAs (current device).
int lookup_shape(const Column &c, uint32_t *parts, uint32_t *grid, uint32_t *resident);
int launch_lookup_rowids(const Column &c, const uint32_t *d_rowids, uint64_t m, int32_t *d_out, cudaStream_t s);

// Fused conjunction + lookup (fused.cu): cols[p] with predicate kp[p], p <
// npred (1..4, equal lengths), then the values of `proj` at the selected rows
// in ascending row order; d_bits (optional) also receives the result bit
// vector. d_ws: scan_lookup_workspace_bytes(proj) bytes, cleared by the call.
uint64_t scan_lookup_workspace_bytes(const Column &proj);
int launch_scan_lookup(const Column *const *cols, const KPred *kp, int npred, const Column &proj, uint32_t *d_bits,
                       int32_t *d_out, uint64_t out_cap, uint64_t *d_count, void *d_ws, cudaStream_t s);

int read_and_clear_status(uint32_t *status);
// Device address of the status word on the current device (nullptr on error).
uint32_t *status_word();
int sm_count(int device);
// Resident blocks per SM of a kernel (cached per kernel and device).
int blocks_per_sm(const void *kernel, int threads, size_t smem, int device);

}  // namespace bs
