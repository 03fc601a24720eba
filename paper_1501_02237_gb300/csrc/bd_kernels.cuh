// Device-side declarations shared by the C ABI translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bd_core.cuh"

namespace bd {

// Global accumulators of one enumeration (one system).
struct DevAcc {
  unsigned long long nvol_lo, nvol_hi;  // sum |D0| as unsigned 128-bit
  unsigned long long cells, singular, ties;
  unsigned long long items_done;
};

struct EnumParams {
  const int64_t* pts;     // N x K coordinates, row-major (device)
  const int64_t* lifts;   // N explicit lift heights (device) or nullptr: use (lift_seed, attempt)
  uint64_t lift_seed;     // stream seed (see bd_lifts.h)
  const PackedItem* items;  // the work list (packed prefixes)
  int nitems;
  const Range* ranges;    // work units: ranges of consecutive items, or nullptr: one item each
  int nranges;
  int shard, shards;      // this launch takes the units u with u % shards == shard (shards >= 1)
  int N, K;
  int five;               // 1: the 5-D bottom stage (32-bit coordinate path, K >= 4): the launch
                          // runs that stage's kernel; the work list's depth must agree (item_depth)
  unsigned int* counter;  // next work unit (reset to 0 before the launch)
  const uint32_t* tri;    // colex decode table of kTriEntries words (device), or nullptr
  CellSink sink;          // accepted cells are recorded here when sink.out is non-null
  DevAcc* acc;            // reset to 0 before the launch
};

struct LaunchShape {
  int blocks = 0, warps = 0;
  size_t smem = 0;       // dynamic shared memory per block
  int slots = 0;         // points per warp stack (multiple of 32)
};

// Integer paths: coordinate minors / lift minors in (int32, int64), (int64, int64), (int128, int128)
enum { PATH_NARROW = 0, PATH_MID = 1, PATH_WIDE = 2 };

// Shared memory of one block: lifted points + one stack per warp.
size_t enum_smem_bytes(int N, int K, int warps, int path);
// five: the launch runs the 5-D bottom stage (path PATH_NARROW, K >= 4; EnumParams.five)
LaunchShape enum_shape(int N, int K, int path, bool five, int warps_req, int blocks_per_sm_req, int sms, cudaError_t* err);
cudaError_t launch_enumerate(const EnumParams& p, const LaunchShape& s, int path, cudaStream_t st);

// One warp per given subset: status (0 singular, 1 rejected, 2 accepted, 3 tie) and |D0|.
cudaError_t launch_classify(const int64_t* pts, const int64_t* lifts, int N, int K, const uint8_t* subsets,
                            int count, int32_t* status, int64_t* absdet, int path, cudaStream_t st);

// ---- batches: many systems in one persistent launch ---------------------------------------

constexpr int BATCH_KMAX = 12;  // a batch item keeps 11 prefix indices
constexpr int BD_SERVE_PTS = 64 * BATCH_KMAX;  // coordinates kept per serving slot

struct BatchDesc {       // one system of a batch
  int N, K;
  int pts_off;           // offset of its N x K coordinates in the packed point array
  int path;
  int five;              // 1: the 5-D bottom stage on the 32-bit coordinate path (K >= 4)
  int gen;               // serving: the admission that holds the slot (a slot is reused)
  uint64_t lift_seed;    // stream seed of its current lifting
};
static_assert(sizeof(BatchDesc) % 8 == 0, "descriptors are read as 64-bit words");

struct BatchItem {       // a prefix of one system's subset tree
  uint32_t sys;
  uint8_t len;
  uint8_t idx[11];
};

struct BatchParams {
  const BatchDesc* desc;
  const int64_t* pts;
  const BatchItem* items;
  int nitems;
  int maxN, maxK;                 // shared-memory layout bounds of this launch
  unsigned int* counter;          // next item (reset before the launch)
  DevAcc* acc;                    // per system (reset before the launch)
  unsigned long long* cycles;     // per system: SM cycles spent in its items
  unsigned int* done;             // per system: items finished (for streaming completion)
  const uint32_t* tri;            // colex decode table (device) or nullptr
};

size_t batch_smem_bytes(int maxN, int maxK, int warps, int path);
// five: every system of the launch runs the 5-D bottom stage (path PATH_NARROW, K >= 4); a
// launch carries one stage, so a batch groups its systems by path and stage
LaunchShape batch_shape(int maxN, int maxK, int path, bool five, int warps_req, int blocks_per_sm_req, int sms,
                        cudaError_t* err);
cudaError_t launch_batch(const BatchParams& p, const LaunchShape& s, int path, bool five, cudaStream_t st);

// ---- serving: a persistent kernel fed while it runs ------------------------------------------

struct ServeParams {
  const BatchDesc* desc;            // per slot (device)
  const int64_t* pts;               // per slot: BD_NMAX x BATCH_KMAX coordinates (device)
  const BatchItem* ring;            // work items, index = ticket % ring_cap (device)
  unsigned long long ring_cap;
  unsigned long long* head;         // next ticket to claim (device, fetch-and-add)
  const volatile unsigned long long* tail;  // tickets below tail are published (device, host-written)
  unsigned int* remaining;          // per slot: items not yet finished (device)
  DevAcc* acc;                      // per slot (device)
  unsigned long long* cycles;       // per slot (device)
  unsigned long long* comp_count;   // completions so far (device)
  volatile unsigned long long* comp; // completion records (host-mapped): (sequence << 32) | slot
  volatile unsigned long long* res;  // per slot (host-mapped): its final DevAcc words and SM cycles,
                                     // written before the slot's completion record
  unsigned long long comp_cap;
  const volatile int* stop;         // device: 1 asks every warp waiting for an unpublished
                                    // ticket to exit (server stop)
  unsigned long long idle_ns;       // after this long without a publication, waiting warps give
                                    // their tickets back and exit (the host relaunches on demand)
  const volatile unsigned long long* seq;  // per ring position: ticket + 1 once its item is published (device)
  unsigned long long* fault_dev;    // device: ticket + 1 of the first item whose publication wait ran out
  volatile unsigned long long* fault_host;  // host-mapped copy of fault_dev for the host's pump
  unsigned long long wait_ns;       // bound of the publication wait (globaltimer nanoseconds)
  int maxN, maxK;
  const uint32_t* tri;              // colex decode table (device) or nullptr
};

constexpr int kServeResWords = sizeof(DevAcc) / 8 + 1;  // ServeParams.res words per slot
size_t serve_smem_bytes(int maxN, int maxK, int warps);
LaunchShape serve_shape(int maxN, int maxK, int warps_req, int blocks_per_sm_req, int sms, cudaError_t* err);
cudaError_t launch_serve(const ServeParams& p, const LaunchShape& s, cudaStream_t st);

// The inner normals of `count` recorded cells (16-byte records), one thread per cell:
// den[i] > 0, alpha[i*K + c], beta[2i] (low 64 bits) and beta[2i+1] (high); status[i] = 0 or
// 1 (flat cell or a value out of range).  Lifts: explicit (lifts) or from lift_seed.
cudaError_t launch_cell_normals(const int64_t* pts, const int64_t* lifts, uint64_t lift_seed, int N, int K,
                                const uint8_t* cells, unsigned long long count, int64_t* den, int64_t* alpha,
                                int64_t* beta, int32_t* status, cudaStream_t st);

}  // namespace bd
