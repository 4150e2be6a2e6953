// The device arena the server carves its field sets from (hf::Arena), and
// its bookkeeping self-check (hf_arena_selftest).  Host code only.
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <iterator>
#include <random>
#include <vector>

#include "hf.h"
#include "hf_internal.h"

namespace hf {

namespace {
size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
}  // namespace

void Arena::reset(uintptr_t base, size_t bytes) {
    std::lock_guard<std::mutex> g(mu_);
    base_ = base;
    size_ = bytes;
    free_ = bytes;
    failures_ = 0;
    free_list_.clear();
    live_.clear();
    if (bytes) free_list_[0] = bytes;
}

void *Arena::alloc(size_t bytes) {
    if (bytes == 0) return nullptr;
    const size_t len = round_up(bytes, kAlign);
    const size_t align = len >= kLargeAlign ? kLargeAlign : kAlign;
    std::lock_guard<std::mutex> g(mu_);
    // best fit: the smallest free range that holds the aligned request
    auto best = free_list_.end();
    size_t best_start = 0;
    for (auto it = free_list_.begin(); it != free_list_.end(); ++it) {
        const size_t start = round_up(base_ + it->first, align) - base_;
        if (start < it->first || start - it->first > it->second || it->second - (start - it->first) < len) continue;
        if (best == free_list_.end() || it->second < best->second) {
            best = it;
            best_start = start;
        }
    }
    if (best == free_list_.end()) {
        ++failures_;
        return nullptr;
    }
    const size_t off = best->first, flen = best->second;
    free_list_.erase(best);
    if (best_start > off) free_list_[off] = best_start - off;  // the alignment gap stays free
    const size_t end = best_start + len, fend = off + flen;
    if (fend > end) free_list_[end] = fend - end;
    live_[best_start] = len;
    free_ -= len;
    return reinterpret_cast<void *>(base_ + best_start);
}

bool Arena::release(void *p) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    std::lock_guard<std::mutex> g(mu_);
    if (a < base_ || a >= base_ + size_) return false;
    const size_t off = a - base_;
    auto lv = live_.find(off);
    if (lv == live_.end()) return false;
    size_t start = off, len = lv->second;
    live_.erase(lv);
    free_ += len;
    auto next = free_list_.lower_bound(off);
    if (next != free_list_.end() && next->first == start + len) {  // merge with the range after
        len += next->second;
        next = free_list_.erase(next);
    }
    if (next != free_list_.begin()) {  // and with the range before
        auto prev = std::prev(next);
        if (prev->first + prev->second == start) {
            start = prev->first;
            len += prev->second;
            free_list_.erase(prev);
        }
    }
    free_list_[start] = len;
    return true;
}

bool Arena::owns(const void *p) const {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    std::lock_guard<std::mutex> g(mu_);
    return size_ && a >= base_ && a < base_ + size_;
}

size_t Arena::merged_if_released(const void *p) const {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    std::lock_guard<std::mutex> g(mu_);
    if (a < base_ || a >= base_ + size_) return 0;
    const size_t off = a - base_;
    auto lv = live_.find(off);
    if (lv == live_.end()) return 0;
    size_t len = lv->second;
    auto next = free_list_.lower_bound(off);
    if (next != free_list_.end() && next->first == off + lv->second) len += next->second;
    if (next != free_list_.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) len += prev->second;
    }
    return len;
}

size_t Arena::free_range_containing(const void *p) const {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    std::lock_guard<std::mutex> g(mu_);
    if (a < base_ || a >= base_ + size_) return 0;
    const size_t off = a - base_;
    auto it = free_list_.upper_bound(off);
    if (it == free_list_.begin()) return 0;
    --it;
    return off < it->first + it->second ? it->second : 0;
}

size_t Arena::capacity() const {
    std::lock_guard<std::mutex> g(mu_);
    return size_;
}

size_t Arena::free_bytes() const {
    std::lock_guard<std::mutex> g(mu_);
    return free_;
}

size_t Arena::largest_free() const {
    std::lock_guard<std::mutex> g(mu_);
    size_t m = 0;
    for (const auto &f : free_list_) m = f.second > m ? f.second : m;
    return m;
}

int64_t Arena::failures() const {
    std::lock_guard<std::mutex> g(mu_);
    return failures_;
}

size_t Arena::live_count() const {
    std::lock_guard<std::mutex> g(mu_);
    return live_.size();
}

// Free ranges sorted, disjoint and never adjacent; live ranges disjoint from
// each other and from the free ones, aligned, inside the region; free and
// live lengths adding up to the region and the free count matching.
bool Arena::check() const {
    std::lock_guard<std::mutex> g(mu_);
    std::map<size_t, std::pair<size_t, bool>> all;  // offset -> (length, live)
    size_t fsum = 0, total = 0;
    for (const auto &f : free_list_) {
        if (f.second == 0) return false;
        all[f.first] = {f.second, false};
        fsum += f.second;
    }
    for (const auto &l : live_) {
        if (l.second == 0 || l.second % kAlign) return false;
        const size_t align = l.second >= kLargeAlign ? kLargeAlign : kAlign;
        if ((base_ + l.first) % align) return false;
        if (all.count(l.first)) return false;
        all[l.first] = {l.second, true};
    }
    if (fsum != free_) return false;
    size_t at = 0;
    bool prev_free = false;
    for (const auto &r : all) {
        if (r.first != at) return false;  // a gap or an overlap
        if (!r.second.second && prev_free) return false;  // two free ranges adjacent
        prev_free = !r.second.second;
        at = r.first + r.second.first;
        total += r.second.first;
    }
    return at == size_ && total == size_;
}

}  // namespace hf

extern "C" int64_t hf_arena_selftest(uint64_t seed, size_t bytes, int ops) {
    if (bytes == 0 || ops <= 0) return -1;
    hf::Arena a;
    const uintptr_t base = (uintptr_t)1 << 40;  // never dereferenced
    a.reset(base, bytes);
    std::mt19937_64 rng(seed);
    std::vector<std::pair<void *, size_t>> live;
    for (int i = 0; i < ops; ++i) {
        const bool do_alloc = live.empty() || (rng() % 100) < 55;
        if (do_alloc) {
            // sizes log-uniform from 1 byte to a quarter of the region
            const double u = std::uniform_real_distribution<double>(0.0, 1.0)(rng);
            const size_t b = (size_t)std::max(1.0, std::exp(u * std::log((double)bytes / 4)));
            void *p = a.alloc(b);
            if (p) {
                const uintptr_t q = (uintptr_t)p;
                if (q < base || q + b > base + bytes) return i + 1;
                for (const auto &l : live) {  // disjoint from every live range
                    const uintptr_t s = (uintptr_t)l.first;
                    if (q < s + l.second && s < q + b) return i + 1;
                }
                live.push_back({p, b});
            } else if (a.largest_free() >= hf::Arena::kLargeAlign + b + hf::Arena::kAlign) {
                return i + 1;  // refused although a range with room for any alignment was free
            }
        } else {
            const size_t k = rng() % live.size();
            const size_t merged = a.merged_if_released(live[k].first);
            if (merged < live[k].second) return i + 1;
            if (!a.release(live[k].first)) return i + 1;
            if (a.free_range_containing(live[k].first) != merged) return i + 1;  // the range it predicted
            if (a.merged_if_released(live[k].first) != 0) return i + 1;
            if (a.release(live[k].first)) return i + 1;  // a second release of the same range is refused
            live[k] = live.back();
            live.pop_back();
        }
        if (!a.check()) return i + 1;
    }
    for (const auto &l : live)
        if (!a.release(l.first)) return ops + 1;
    if (!a.check() || a.free_bytes() != bytes || a.largest_free() != bytes || a.live_count() != 0) return ops + 2;
    return 0;
}
