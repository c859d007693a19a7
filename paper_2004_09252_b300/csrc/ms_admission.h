// Admission policy of the served form, in plain C++ (no CUDA), so that the
// host logic can be tested on its own.
//
// State: a ring of S staging slots (waves take contiguous runs of slots and
// are released in the order they were issued) and a per-page mark of the
// pages that belong to an admitted, not yet completed wave.
//
// form(): queued requests are scanned in arrival order (at most `window` of
// them) and admitted into one wave while the wave and the ring have room:
//   - a request with a page already in flight (or in this wave) is skipped,
//     and its pages are blocked for the rest of the scan, so a later request
//     that shares one of them cannot overtake it;
//   - running out of ring room ends the scan (no overtaking for room, so a
//     large request is not starved by small ones);
//   - in one-per-launch mode a wave holds one request.
// A wave that does not fit before the end of the ring starts at slot 0, and
// the skipped tail counts as used until the wave is released.
//
// form_inplace(): a wave that takes no staging slots (it runs in place on the
// working set), formed only while the whole queue holds at most max_pages
// pages: every queued request whose pages are free joins it, in arrival
// order, under the same blocking rule.  Its release frees no slots, so such
// waves may be released in any order.
#pragma once

#include <algorithm>
#include <cstdint>
#include <deque>
#include <vector>

namespace ms {

// Per-page marks, two bits a page: in flight (in an admitted, not yet
// completed wave) and blocked (skipped earlier in the current scan).  As
// bitsets the marks of a 16 GiB working set (4M pages) take 1 MiB, so the
// scans of a large wave stay in cache (a byte a page took 4 MiB, and random
// accesses to it cost the server thread milliseconds per large wave).
class PageMarks {
 public:
  explicit PageMarks(uint64_t n) : busy_((n + 63) / 64, 0), blocked_((n + 63) / 64, 0) {}
  bool taken(uint64_t pg) const { return ((busy_[pg >> 6] | blocked_[pg >> 6]) >> (pg & 63)) & 1u; }
  void set_busy(uint64_t pg) { busy_[pg >> 6] |= bit(pg); }
  void clear_busy(uint64_t pg) { busy_[pg >> 6] &= ~bit(pg); }
  void set_blocked(uint64_t pg) { blocked_[pg >> 6] |= bit(pg); }
  void clear_blocked(uint64_t pg) { blocked_[pg >> 6] &= ~bit(pg); }

 private:
  static uint64_t bit(uint64_t pg) { return 1ull << (pg & 63); }
  std::vector<uint64_t> busy_, blocked_;
};

struct AdmittedWave {
  std::vector<uint64_t> tickets;
  uint32_t pos = 0;   // first staging slot
  uint32_t len = 0;   // pages
  uint32_t span = 0;  // ring slots consumed: len plus the skipped tail
};

class Admission {
 public:
  Admission(uint32_t slots, uint32_t max_wave_pages, bool one_per_launch, uint64_t n_pages, size_t window)
      : S_(slots), max_wave_(max_wave_pages), one_(one_per_launch), window_(window), marks_(n_pages) {}

  uint32_t slots() const { return S_; }
  uint32_t used() const { return used_; }
  uint64_t conflict_waits = 0, budget_waits = 0;

  // pages_of(ticket) returns the request's page list (a container of uint64_t).
  // The cost is proportional to the requests scanned, not to the queue: a
  // one-request wave taken from a long backlog touches only the head.
  template <typename PagesOf>
  bool form(std::deque<uint64_t> &queue, PagesOf pages_of, AdmittedWave &w) {
    if (used_ == 0) head_ = 0;  // nothing in flight: the whole ring is free from slot 0
    uint32_t pos = head_, waste = 0, len = 0;
    const size_t window = std::min(queue.size(), window_);
    std::vector<uint8_t> taken;  // one flag per scanned request
    std::vector<uint64_t> blocked;
    size_t n_taken = 0;
    for (size_t i = 0; i < window; ++i) {
      const auto &pages = pages_of(queue[i]);
      const uint32_t n = (uint32_t)pages.size();
      if (one_ && n_taken == 1) break;
      if (len + n > max_wave_ && n_taken > 0) break;
      uint32_t p = pos, wst = waste;
      if (len == 0 && p + n > S_) {  // wrap to slot 0
        wst = S_ - p;
        p = 0;
      }
      if (p + len + n > S_ || used_ + wst + len + n > S_) {
        ++budget_waits;
        break;
      }
      bool conflict = false;
      for (uint64_t pg : pages)
        if (marks_.taken(pg)) {
          conflict = true;
          break;
        }
      if (conflict) {
        ++conflict_waits;
        for (uint64_t pg : pages)
          if (!marks_.taken(pg)) {
            marks_.set_blocked(pg);  // blocked for the rest of this scan
            blocked.push_back(pg);
          }
        taken.push_back(0);
        continue;
      }
      for (uint64_t pg : pages) marks_.set_busy(pg);
      pos = p;
      waste = wst;
      len += n;
      w.tickets.push_back(queue[i]);
      taken.push_back(1);
      ++n_taken;
    }
    for (uint64_t pg : blocked) marks_.clear_blocked(pg);
    if (n_taken == 0) return false;
    // drop the admitted tickets from the scanned prefix, keeping the skipped ones in order
    const size_t scanned = taken.size();
    std::vector<uint64_t> keep;
    keep.reserve(scanned - n_taken);
    for (size_t i = 0; i < scanned; ++i)
      if (!taken[i]) keep.push_back(queue[i]);
    queue.erase(queue.begin(), queue.begin() + (long)scanned);
    for (size_t i = keep.size(); i-- > 0;) queue.push_front(keep[i]);
    w.pos = pos;
    w.len = len;
    w.span = waste + len;
    head_ = pos + len;
    used_ += w.span;
    return true;
  }

  // A wave for the in-place lane (see the top of the file): false when the
  // queue holds more than max_pages pages or nothing can be admitted.
  template <typename PagesOf>
  bool form_inplace(std::deque<uint64_t> &queue, PagesOf pages_of, AdmittedWave &w, uint32_t max_pages) {
    if (queue.empty() || queue.size() > max_pages) return false;
    uint32_t total = 0;
    for (uint64_t t : queue) total += (uint32_t)pages_of(t).size();
    if (total > max_pages) return false;
    std::vector<uint64_t> blocked, keep;
    uint32_t len = 0;
    for (uint64_t t : queue) {
      const auto &pages = pages_of(t);
      bool conflict = false;
      for (uint64_t pg : pages)
        if (marks_.taken(pg)) {
          conflict = true;
          break;
        }
      if (conflict) {
        ++conflict_waits;
        for (uint64_t pg : pages)
          if (!marks_.taken(pg)) {
            marks_.set_blocked(pg);
            blocked.push_back(pg);
          }
        keep.push_back(t);
        continue;
      }
      for (uint64_t pg : pages) marks_.set_busy(pg);
      len += (uint32_t)pages.size();
      w.tickets.push_back(t);
    }
    for (uint64_t pg : blocked) marks_.clear_blocked(pg);
    if (w.tickets.empty()) return false;
    queue.assign(keep.begin(), keep.end());
    w.pos = 0;
    w.len = len;
    w.span = 0;
    return true;
  }

  // A completed wave: its pages leave the in-flight set and its slots are
  // freed.  Waves with slots must be released in the order form() returned
  // them; in-place waves (span 0) in any order.
  template <typename PagesOf>
  void release(const AdmittedWave &w, PagesOf pages_of) {
    for (uint64_t t : w.tickets)
      for (uint64_t pg : pages_of(t)) marks_.clear_busy(pg);
    used_ -= w.span;
  }

 private:
  uint32_t S_, max_wave_;
  bool one_;
  size_t window_;
  PageMarks marks_;
  uint32_t head_ = 0, used_ = 0;
};

}  // namespace ms
