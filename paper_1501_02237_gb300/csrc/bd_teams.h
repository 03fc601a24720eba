// Host stand-ins for a warp: a one-lane team, and a team of `width` lanes run as CPU threads
// in lockstep, so that the warp-synchronous walkers run unchanged in the host emulation.
#pragma once

#include <condition_variable>
#include <cstdint>
#include <mutex>
#include <vector>

namespace bd {

struct HostTeam {
  int lane() const { return 0; }
  int lanes() const { return 1; }
  bool any(bool b) const { return b; }
  bool all(bool b) const { return b; }
  void sync() const {}
  uint64_t or_all(uint64_t x) const { return x; }
  uint32_t max_u32(uint32_t x) const { return x; }
  uint64_t ballot(bool b) const { return b ? 1ull : 0ull; }
};

// A team of `width` lanes run as CPU threads in lockstep: every collective (vote, sync) is a
// barrier, as a warp-synchronous program requires of its lanes.  Tests use it to run the
// multi-lane logic of the walker (lane dealing, ragged tails, votes) without a GPU.
struct LockstepShared {
  std::mutex mu;
  std::condition_variable cv;
  int width, waiting = 0;
  uint64_t generation = 0;
  std::vector<uint64_t> votes;
  explicit LockstepShared(int w) : width(w), votes(w) {}
  void barrier() {
    std::unique_lock<std::mutex> lk(mu);
    const uint64_t g = generation;
    if (++waiting == width) {
      waiting = 0;
      ++generation;
      cv.notify_all();
    } else {
      cv.wait(lk, [&] { return generation != g; });
    }
  }
};

struct LockstepTeam {
  LockstepShared* sh;
  int ln;
  int lane() const { return ln; }
  int lanes() const { return sh->width; }
  uint64_t reduce_or(uint64_t x, bool all_of) const {
    sh->votes[ln] = x;
    sh->barrier();
    uint64_t r = all_of ? 1 : 0;
    for (int w = 0; w < sh->width; ++w) r = all_of ? (r & (sh->votes[w] != 0)) : (r | sh->votes[w]);
    sh->barrier();
    return r;
  }
  bool any(bool b) const { return reduce_or(b, false) != 0; }
  uint64_t ballot(bool b) const { return reduce_or(b ? 1ull << ln : 0ull, false); }  // bit l: lane l's vote
  bool all(bool b) const { return reduce_or(b, true) != 0; }
  void sync() const { sh->barrier(); }
  uint64_t or_all(uint64_t x) const { return reduce_or(x, false); }
  uint32_t max_u32(uint32_t x) const {
    sh->votes[ln] = x;
    sh->barrier();
    uint64_t r = 0;
    for (int w = 0; w < sh->width; ++w) r = sh->votes[w] > r ? sh->votes[w] : r;
    sh->barrier();
    return (uint32_t)r;
  }
};

}  // namespace bd
