// Bounded cache of captured CUDA graphs, keyed by a call's arguments.
//
// bits_mc, bits_count_matrix and bits_mc_matrix capture their launches once
// per argument set and replay the graph when the same arguments come back.
// A caller that sweeps seeds, shuffle ranges or output buffers would
// otherwise keep one graph (and its small device buffers) per argument set
// for the life of the database; here at most `cap` graphs stay cached and
// the least recently used one is dropped first.  Dropping a graph first
// waits for the device to finish (its executable and device buffers may
// still be in use by a replay in flight).
#pragma once

#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <utility>

#include "common.cuh"

namespace bits {

template <class Key, class G>
class GraphCache {
 public:
  explicit GraphCache(size_t cap) : cap_(cap) {}

  // The cached graph of `k` (marked most recently used), or null.
  std::shared_ptr<G> find(const Key& k) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = index_.find(k);
    if (it == index_.end()) return nullptr;
    order_.splice(order_.begin(), order_, it->second);
    return it->second->second;
  }

  // Cache g under k, dropping the least recently used graphs beyond the cap.
  void put(const Key& k, std::shared_ptr<G> g) {
    std::list<std::shared_ptr<G>> dropped;
    {
      std::lock_guard<std::mutex> lk(mu_);
      auto it = index_.find(k);
      if (it != index_.end()) {
        it->second->second = std::move(g);
        order_.splice(order_.begin(), order_, it->second);
        return;
      }
      order_.emplace_front(k, std::move(g));
      index_[k] = order_.begin();
      while (order_.size() > cap_) {
        dropped.push_back(std::move(order_.back().second));
        index_.erase(order_.back().first);
        order_.pop_back();
      }
    }
    if (!dropped.empty()) cudaDeviceSynchronize();
    dropped.clear();
  }

  // Drop every graph whose key satisfies pred (e.g. one that names a
  // database being freed); the caller has synchronised the device.
  template <class Pred>
  void erase_if(Pred pred) {
    std::lock_guard<std::mutex> lk(mu_);
    for (auto it = order_.begin(); it != order_.end();) {
      if (pred(it->first)) {
        index_.erase(it->first);
        it = order_.erase(it);
      } else {
        ++it;
      }
    }
  }

  size_t size() {
    std::lock_guard<std::mutex> lk(mu_);
    return order_.size();
  }

 private:
  size_t cap_;
  std::mutex mu_;
  std::list<std::pair<Key, std::shared_ptr<G>>> order_;
  std::map<Key, typename std::list<std::pair<Key, std::shared_ptr<G>>>::iterator> index_;
};

}  // namespace bits
