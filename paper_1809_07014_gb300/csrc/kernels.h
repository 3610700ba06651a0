// Launchers of the device kernels (host side of each .cu file).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"

namespace kmer {

// A kernel's dynamic shared-memory limit is one attribute per function and
// device, shared by every host thread: raise it to `bytes` when it is lower,
// never lower it (a thread that lowered it could make another thread's launch
// with a larger size fail).  The limits set are remembered per process; a
// cudaDeviceReset() by the application clears the attributes but not this
// record, so such an application must not reset a device it still analyses on.
inline cudaError_t raise_smem_limit(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = limit[{dev, func}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

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

// A fallback list entry: a leaf and the key range of it to recount in HBM,
// the records whose next `rb` z bits (below the leaf's) equal `rs`.
constexpr unsigned kFbLeafBits = 22;
__host__ __device__ inline unsigned fallback_entry(unsigned leaf, unsigned rb, unsigned rs) {
    return leaf | (rb << kFbLeafBits) | (rs << (kFbLeafBits + 3));
}
__host__ __device__ inline unsigned fallback_leaf(unsigned e) { return e & ((1u << kFbLeafBits) - 1u); }
__host__ __device__ inline unsigned fallback_rb(unsigned e) { return (e >> kFbLeafBits) & 7u; }
__host__ __device__ inline unsigned fallback_rs(unsigned e) { return e >> (kFbLeafBits + 3); }

// All three stages take a device array of Job descriptors (all of key width
// W) and work over every job of the array in one launch.

// Index of the survivors (positions in an open-addressing table of `cap`
// slots, all 0xFFFFFFFF before the build) for point lookups (lookup.cu).
cudaError_t launch_index_build(unsigned W, const unsigned long long* keys, unsigned long long n, unsigned* idx,
                               unsigned long long cap, int num_sms, cudaStream_t s);

// Bloom gate (gate.cu): adds every window's key of the job's reads to filter
// f1, and keys already in f1 to f2 (both 2^log2_words words, zeroed by the
// caller); counts[0..2] += windows, first sightings, keys entering f2.
cudaError_t launch_gate(const Job& j, unsigned long long* f1, unsigned long long* f2, unsigned log2_words,
                        unsigned long long* counts, cudaStream_t s);

// Merge (Algorithm 1): k-mers of a second canonical, distinct set (bkeys,
// bcls; bn of them) absent from the indexed survivors are appended to them
// from position *n_out on (count 0, zero tallies, their own classes); a
// position past out_cap sets bit 0 of *status.
// Pieces of a byte string: piece i is src[psrc[i] ..) of pdst[i + 1] - pdst[i]
// bytes, written to dst[pdst[i] ..) (pdst: n_pieces + 1 offsets).
cudaError_t launch_piece_copy(const char* src, const unsigned long long* psrc, const unsigned long long* pdst,
                              unsigned long long n_pieces, char* dst, int num_sms, cudaStream_t s);
cudaError_t launch_merge_append(unsigned W, const unsigned long long* bkeys, const unsigned char* bcls,
                                unsigned long long bn, const unsigned* idx, unsigned long long cap,
                                unsigned long long* keys, unsigned* count, unsigned* ext, unsigned char* cls,
                                unsigned long long out_cap, unsigned long long* n_out, unsigned* status, int num_sms,
                                cudaStream_t s);

// De Bruijn graph traversal (traverse.cu) over n survivors (keys, classes)
// with their index: plan (links, list ranking, rings, lengths; totals[0] =
// contig bases, totals[1] = contigs, device), then write (contig bases into
// out, contig_off = n_contigs + 1 offsets).  scratch: traverse_scratch_bytes,
// kept between the two calls.
size_t traverse_scratch_bytes(unsigned long long n);
cudaError_t launch_traverse_plan(unsigned W, const unsigned long long* keys, const unsigned char* cls,
                                 unsigned long long n, unsigned k, const unsigned* idx, unsigned long long cap,
                                 void* scratch, unsigned long long* totals, int num_sms, cudaStream_t s);
cudaError_t launch_traverse_write(unsigned W, const unsigned long long* keys, const unsigned char* cls,
                                  unsigned long long n, unsigned k, unsigned long long n_contigs, void* scratch,
                                  char* out, unsigned long long* contig_off, int num_sms, cudaStream_t s);

// Survivors in ascending key order: LSD radix sort of the n keys (8-bit
// digits over the 2k key bits, one-sweep passes, n < 2^32), then count / ext /
// cls gathered through the permutation; all four arrays are rewritten in
// place.  scratch: sort_scratch_bytes; *launches counts the kernels; status
// gets ST_TIMEOUT if a look-back gave up and ST_SORT_RANGE if a position fell
// outside [0, n) (its write skipped).  Synchronises the stream once (to skip
// passes whose digit is constant).
size_t sort_scratch_bytes(unsigned W, unsigned long long n);
cudaError_t launch_sort_survivors(unsigned W, unsigned long long* keys, unsigned* count, unsigned* ext,
                                  unsigned char* cls, unsigned long long n, unsigned k, void* scratch,
                                  unsigned* status, int num_sms, unsigned* launches, cudaStream_t s);

// Level-1 scatter (a2-a3 + partition): one CTA per read tile of 256 reads;
// tile_off = exclusive prefix (n_jobs + 1) of the jobs' read tiles; min_k =
// the smallest k of the jobs (one-word keys with k >= 17 roll on their high
// half).
size_t scatter_smem_bytes(unsigned W, unsigned p1);
// gated: every job carries a Bloom gate (Job::gate) and emits only its keys.
cudaError_t launch_scatter(unsigned W, const Job* jobs, const unsigned long long* tile_off, unsigned n_jobs,
                           unsigned long long tiles, unsigned max_p1, unsigned min_k, bool gated, cudaStream_t s);

// Per analysis: level-2 tile counts, leaf capacities and leaf region bases;
// then job_tile_off = prefix of the analyses' level-2 tiles (device array).
cudaError_t launch_l2_plan(const Job* jobs, unsigned n_jobs, unsigned long long* job_tile_off, cudaStream_t s);
// Level-2 repartition of every level-1 bucket of every analysis into its leaves.
size_t repart_smem_bytes(unsigned W, unsigned p2);
cudaError_t launch_repart(unsigned W, const Job* jobs, const unsigned long long* job_tile_off, unsigned n_jobs,
                          unsigned max_p2, int num_sms, cudaStream_t s);

// a4-a7 fused: count each leaf in shared memory, filter, classify, compact;
// leaf_off = exclusive prefix (n_jobs + 1) of the analyses' leaf counts.
unsigned leaf_table_cap(unsigned W, size_t smem_budget);
size_t leaf_smem_bytes(unsigned W, unsigned cap);
// Leaves listed in each analysis's split list, counted in key ranges (after
// launch_leaf, same shared-memory table).
cudaError_t launch_leaf_split(unsigned W, const Job* jobs, unsigned n_jobs, unsigned cap_max, int num_sms,
                              cudaStream_t s);
cudaError_t launch_leaf(unsigned W, const Job* jobs, const unsigned long long* leaf_off, unsigned n_jobs,
                        unsigned long long leaves, unsigned cap_max, int num_sms, cudaStream_t s);

// HBM open-addressing table (direct variant and fallback for leaves that do
// not fit on chip).  Entries are zeroed by the caller (cudaMemsetAsync 0).
size_t hbm_entry_bytes(unsigned W);
cudaError_t launch_direct_insert(const Job& j, void* table, unsigned long long cap, cudaStream_t s);
cudaError_t launch_records_insert(const Job& j, unsigned entry, void* table, unsigned long long cap, int num_sms,
                                  cudaStream_t s);
cudaError_t launch_hbm_sweep(const Job& j, const void* table, unsigned long long cap, int num_sms, cudaStream_t s);

}  // namespace kmer
