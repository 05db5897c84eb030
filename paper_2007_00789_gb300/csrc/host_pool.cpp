// Host worker threads shared by the library's parallel host loops (the
// symbolic analysis, the pack map, host copies of the input).  The threads are
// started on first use and kept, so that a loop costs a wake-up rather than
// the creation of its threads.
#include <unistd.h>

#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>

#include "spand_internal.h"

namespace spand {
namespace {

struct HostPool {
  explicit HostPool(pid_t p) : pid(p) {}
  const pid_t pid;
  std::mutex job;  // one loop at a time
  std::mutex m;
  std::condition_variable wake, idle;
  const std::function<void(int)>* fn = nullptr;
  uint64_t gen = 0;  // loops started
  int want = 0, taken = 0, done = 0, nthreads = 0;

  void worker() {
    uint64_t seen = 0;
    std::unique_lock<std::mutex> g(m);
    for (;;) {
      wake.wait(g, [&] { return gen != seen; });
      seen = gen;
      if (taken >= want) continue;  // the loop asked for fewer threads
      const int w = 1 + taken++;
      const std::function<void(int)>* f = fn;
      g.unlock();
      (*f)(w);
      g.lock();
      if (++done == want) idle.notify_one();
    }
  }

  bool run(int nth, const std::function<void(int)>& f) {
    std::unique_lock<std::mutex> busy(job, std::try_to_lock);
    if (!busy.owns_lock()) return false;
    {
      std::lock_guard<std::mutex> g(m);
      for (; nthreads < nth - 1; ++nthreads) std::thread(&HostPool::worker, this).detach();
      fn = &f;
      want = nth - 1;
      taken = 0;
      done = 0;
      ++gen;
    }
    wake.notify_all();
    f(0);
    std::unique_lock<std::mutex> g(m);
    idle.wait(g, [&] { return done == want; });
    fn = nullptr;
    return true;
  }
};

}  // namespace

bool host_pool_run(int nth, const std::function<void(int)>& work) {
  static std::mutex mk;
  static HostPool* pool = nullptr;
  HostPool* p;
  {
    std::lock_guard<std::mutex> g(mk);
    // the pool lives as long as the process (its threads wait on it); a forked
    // child, which has none of the parent's threads, starts a pool of its own
    const pid_t pid = getpid();
    if (!pool || pool->pid != pid) pool = new HostPool(pid);
    p = pool;
  }
  return p->run(nth, work);
}

}  // namespace spand
