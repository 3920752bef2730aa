// Host-only policy of the lattice server: a first-fit arena allocator for job workspaces and
// the admission / chunking scheduler.  No CUDA here, so the policy is unit-tested on the CPU.
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <deque>
#include <iterator>
#include <map>
#include <vector>

namespace lbm_serve {

// First-fit allocator over [0, size) in units of `align` bytes; adjacent free blocks coalesce.
class Arena {
  public:
    explicit Arena(size_t size = 0, size_t align = 256) : align_(align), size_(size / align * align) {
        if (size_) free_[0] = size_;
    }
    // Offset of a block of `bytes` (rounded up to the alignment), or -1 if no free block fits.
    int64_t alloc(size_t bytes) {
        const size_t need = (std::max<size_t>(bytes, 1) + align_ - 1) / align_ * align_;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > need) free_[off + need] = len - need;
            used_[off] = need;
            return (int64_t)off;
        }
        return -1;
    }
    // Return a block; false if `off` is not the start of a live block.
    bool release(int64_t off) {
        auto u = used_.find((size_t)off);
        if (u == used_.end()) return false;
        size_t start = u->first, len = u->second;
        used_.erase(u);
        auto next = free_.lower_bound(start);
        if (next != free_.end() && start + len == next->first) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
        return true;
    }
    size_t size() const { return size_; }
    size_t used_bytes() const {
        size_t s = 0;
        for (const auto& kv : used_) s += kv.second;
        return s;
    }
    size_t largest_free() const {
        size_t m = 0;
        for (const auto& kv : free_) m = std::max(m, kv.second);
        return m;
    }
    size_t free_blocks() const { return free_.size(); }
    const std::map<size_t, size_t>& free_list() const { return free_; }
    const std::map<size_t, size_t>& used_list() const { return used_; }

  private:
    size_t align_, size_;
    std::map<size_t, size_t> free_, used_;  // offset -> length
};

enum Policy { kFCFS = 0, kShortestFirst = 1 };

struct JobSpec {
    int64_t id;
    int64_t cells;   // lattice updates per step
    int64_t tiles;   // tiles of the job's step grid
    int64_t steps;   // steps the job asks for
    size_t bytes;    // workspace bytes
};

struct Admit {
    int64_t id;
    int64_t offset;  // workspace offset in the arena
};

// Admission: jobs wait in a queue; a job is admitted while the active set stays within
// max_jobs jobs, max_cells cells and max_tiles tiles and its workspace fits in the arena (a job
// alone may exceed max_cells).  FCFS admits strictly in arrival order (a job that does not fit
// blocks those behind it); kShortestFirst admits the queued job with the least remaining work
// (cells x steps) first, skipping jobs that do not fit.  Every active job advances by the same
// number of steps per round: the chunk, cut so that no job overshoots its step count.
class Scheduler {
  public:
    Scheduler(Policy policy, int max_jobs, int64_t max_cells, int64_t max_tiles, size_t arena_bytes)
        : policy_(policy), max_jobs_(max_jobs), max_cells_(max_cells), max_tiles_(max_tiles), arena_(arena_bytes) {}

    // false if the job can never run (workspace larger than the arena, or more tiles than
    // max_tiles, or no steps)
    bool submit(const JobSpec& j) {
        if (j.bytes > arena_.size() || j.tiles > max_tiles_ || j.steps < 1 || j.cells < 1) return false;
        queue_.push_back(j);
        return true;
    }

    std::vector<Admit> admit() {
        std::vector<Admit> out;
        while (!queue_.empty() && (int)active_.size() < max_jobs_) {
            size_t pick = 0;
            if (policy_ == kShortestFirst) {
                bool found = false;
                for (size_t k = 0; k < queue_.size(); ++k) {
                    if (!fits(queue_[k])) continue;
                    if (!found || work(queue_[k]) < work(queue_[pick])) pick = k;
                    found = true;
                }
                if (!found) break;
            } else if (!fits(queue_[0])) {
                break;
            }
            const JobSpec j = queue_[pick];
            const int64_t off = arena_.alloc(j.bytes);
            if (off < 0) break;  // fragmentation: wait for a release
            queue_.erase(queue_.begin() + (std::ptrdiff_t)pick);
            active_[j.id] = Active{j, 0, off};
            cells_ += j.cells;
            tiles_ += j.tiles;
            out.push_back(Admit{j.id, off});
        }
        return out;
    }

    // Steps of the next round: chunk, or fewer if an active job has fewer left (0 if idle).
    int64_t next_chunk(int64_t chunk) const {
        int64_t n = 0;
        for (const auto& kv : active_) {
            const int64_t left = kv.second.spec.steps - kv.second.done;
            n = n == 0 ? std::min(chunk, left) : std::min(n, left);
        }
        return n;
    }

    // All active jobs advanced by n steps; returns the finished ones (their memory released).
    std::vector<int64_t> advance(int64_t n) {
        std::vector<int64_t> fin;
        for (auto it = active_.begin(); it != active_.end();) {
            it->second.done += n;
            if (it->second.done >= it->second.spec.steps) {
                fin.push_back(it->first);
                finish(it->second);
                it = active_.erase(it);
            } else {
                ++it;
            }
        }
        return fin;
    }

    // Remove an active job early (failure); false if it is not active.
    bool cancel(int64_t id) {
        auto it = active_.find(id);
        if (it == active_.end()) return false;
        finish(it->second);
        active_.erase(it);
        return true;
    }

    bool idle() const { return active_.empty(); }
    size_t queued() const { return queue_.size(); }
    size_t active_count() const { return active_.size(); }
    int64_t active_cells() const { return cells_; }
    int64_t active_tiles() const { return tiles_; }
    std::vector<int64_t> active_ids() const {
        std::vector<int64_t> ids;
        for (const auto& kv : active_) ids.push_back(kv.first);
        return ids;
    }
    int64_t steps_done(int64_t id) const {
        auto it = active_.find(id);
        return it == active_.end() ? -1 : it->second.done;
    }
    const Arena& arena() const { return arena_; }

  private:
    struct Active {
        JobSpec spec;
        int64_t done;
        int64_t offset;
    };
    static double work(const JobSpec& j) { return (double)j.cells * (double)j.steps; }
    bool fits(const JobSpec& j) const {
        if (active_.empty()) return true;
        return cells_ + j.cells <= max_cells_ && tiles_ + j.tiles <= max_tiles_;
    }
    void finish(const Active& a) {
        arena_.release(a.offset);
        cells_ -= a.spec.cells;
        tiles_ -= a.spec.tiles;
    }

    Policy policy_;
    int max_jobs_;
    int64_t max_cells_, max_tiles_;
    Arena arena_;
    std::deque<JobSpec> queue_;
    std::map<int64_t, Active> active_;
    int64_t cells_ = 0, tiles_ = 0;
};

}  // namespace lbm_serve
