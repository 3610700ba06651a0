// Launchers of the device kernels (host side of each .cu file).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace kmer {

constexpr int kLenExact = 128;            // read lengths below this are histogrammed exactly
constexpr int kLenHist = kLenExact + 2;   // + count and sum of longer reads

size_t scan_temp_bytes(unsigned long long n);
cudaError_t exclusive_scan_u64(const unsigned long long* in, unsigned long long* out, unsigned long long n,
                               void* temp, cudaStream_t s);

cudaError_t launch_read_geometry(const unsigned long long* offsets, unsigned long long n, unsigned long long* nblk,
                                 unsigned long long* len_stats, unsigned int* bad, cudaStream_t s);
cudaError_t launch_pack(const char* bases, const unsigned char* quals, const unsigned long long* offsets,
                        const unsigned long long* blk_off, unsigned long long n, unsigned qual_offset,
                        unsigned qual_threshold, PackedBlock* out, int num_sms, cudaStream_t s);

// Level-1 scatter (a2-a3 + partition): every window of reads [r0, r1) of the job.
size_t scatter_smem_bytes(unsigned W, unsigned p1);
cudaError_t launch_scatter(const Job& j, unsigned long long r0, unsigned long long r1, cudaStream_t s);

// Per bucket: level-2 tile counts, leaf capacities and leaf region bases.
cudaError_t launch_l2_plan(const Job& j, unsigned long long l2_capacity, cudaStream_t s);
// Level-2 repartition of every level-1 bucket into its leaves.
size_t repart_smem_bytes(unsigned W, unsigned p2);
cudaError_t launch_repart(const Job& j, int num_sms, cudaStream_t s);

// a4-a7 fused: count each leaf in shared memory, filter, classify, compact.
unsigned leaf_table_cap(unsigned W, size_t smem_budget);
size_t leaf_smem_bytes(unsigned W, unsigned cap);
cudaError_t launch_leaf(const Job& j, unsigned cap_max, int num_sms, cudaStream_t s);

// HBM open-addressing table (direct variant and fallback for leaves that do
// not fit on chip).  Entries are zeroed by the caller (cudaMemsetAsync 0).
size_t hbm_entry_bytes(unsigned W);
cudaError_t launch_direct_insert(const Job& j, void* table, unsigned long long cap, cudaStream_t s);
cudaError_t launch_records_insert(const Job& j, unsigned leaf, void* table, unsigned long long cap, int num_sms,
                                  cudaStream_t s);
cudaError_t launch_hbm_sweep(const Job& j, const void* table, unsigned long long cap, int num_sms, cudaStream_t s);

}  // namespace kmer
