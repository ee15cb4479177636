// rqa_kernels.h -- host-side entry points of the CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "rqa_internal.h"

namespace rqa {

using TileFn = void (*)(const SeriesDesc*, const Item*, int, int*);

// A caller's device pointer that kernels will read: RQA_OK if it is `align`-
// byte aligned and CUDA reports memory that `device` can read (its own
// device memory, managed memory, or mapped pinned host memory), else
// RQA_EINVAL with *what_failed set to a static description.  A misaligned
// or host pointer would otherwise fault the device.
int check_device_pointer(const void* p, size_t align, int device, const char** what_failed);

// Fused tile kernel for embedding dimension m (1..10), norm (0 max, 1 L2,
// 2 L1), columns per lane `cols` (4), FP64-everywhere or FP32 + recheck, and
// the symmetric (RQA) or cross-recurrence matrix, with or without row bands.
TileFn tile_kernel_for(int m, int norm, int cols, bool f64, bool cross, bool bands = false);
size_t tile_smem_for(int m, int norm, bool f64, int warps, int cols);

TileFn tile_kernel_norm0(int m, int cols, bool f64, bool bands);
TileFn tile_kernel_norm1(int m, int cols, bool f64, bool bands);
TileFn tile_kernel_norm2(int m, int cols, bool f64, bool bands);
TileFn tile_kernel_cross_norm0(int m, int cols, bool f64, bool bands);
TileFn tile_kernel_cross_norm1(int m, int cols, bool f64, bool bands);
TileFn tile_kernel_cross_norm2(int m, int cols, bool f64, bool bands);
// The test instantiation of the bounded ring waits: m = 3, L2, four
// columns per lane, FP32 + recheck, RQA, no row bands, a short wait limit.
TileFn tile_kernel_wait_test();
// Line detection over a precomputed bit matrix (no distances).
TileFn tile_kernel_matrix(int cols, bool bands = false);

// max_len: the longest series (both series for cross recurrence) of the set
void launch_prepare(SeriesDesc* d_sd, int count, int64_t max_len, int sms, cudaStream_t st);
void launch_embed(SeriesDesc* d_sd, int count, int64_t max_n_mp, int sms, cudaStream_t st);
// The merge and finalize kernels; `sym` / `cross` say whether the set holds
// RQA series (rows, diagonals, line-of-identity join) and cross-recurrence
// series (diagonals of the rectangle), `bands` whether an RQA series runs in
// row bands (column joins); max_n bounds the rows, columns and diagonals of
// any series.  Returns the number of kernels launched.
int launch_merges(SeriesDesc* d_sd, int count, int64_t max_n, bool sym, bool cross, bool bands,
                  int sms, cudaStream_t st, bool grouped = false);
// A single RQA series run in strip groups: the row and diagonal merges of
// strips q0 .. q1 (carries in rcarry / dcarry); launch_merges(..., grouped)
// then does the rest after the last group.  Returns the kernels launched.
int launch_group_merges(SeriesDesc* d_sd, int64_t n, int64_t q0, int64_t q1, int sms,
                        cudaStream_t st);
void launch_plot(const SeriesDesc* d_sd, int64_t i0, int64_t j0, int64_t rows, int64_t cols,
                 uint32_t* out, int f64, int m, int norm, int sms, cudaStream_t st);
// Bounded-wait self-test (status[3] in device memory: status, cycles, abort).
void launch_wait_selftest(unsigned long long* status, cudaStream_t st);
// Load every kernel of the library into the current context (see
// rqa_preload_kernels); the count loaded, or -1 on a CUDA error.
int preload_tile_kernels();
int preload_aux_kernels();
// Resolves the address of rqa_run_noalloc's static scratch on the current
// device and loads its kernel (1, or -1 on a CUDA error).
int preload_noalloc();
void launch_sample(const SeriesDesc* d_sd, const int64_t* ii, const int64_t* jj, int64_t count,
                   uint8_t* out, int f64, cudaStream_t st);

}  // namespace rqa
