// pool.cu -- the host thread pool behind parallel_for.
//
// The host planners split work over up to 16 threads: the learned plan's
// feature rows, and the block planner's search of qubit triples, once per
// growth step.  Starting threads per call cost about 0.3 ms for 8 threads,
// as much as the work of one triple search, so the threads are started
// once and kept.
//
// A call posts a job (count, function, context) to a queue, wakes the
// workers, and takes indices from the job itself until none are left.  So
// the caller can always finish the job alone: a worker that is busy, asleep
// or missing can slow it but never block it.  This matters for a call made
// from inside a job (it runs serially in a worker, and as a nested job from
// the calling thread), for several host threads calling at once, and for a
// child process forked while the pool was idle (it has no workers).  The
// caller then waits until every worker that took the job has left it,
// because the job lives on the caller's stack.  The pool is never destroyed;
// its threads end with the process.
#include <condition_variable>
#include <deque>
#include <mutex>

#include "internal.cuh"

namespace qsim {

namespace {

struct Job {
    size_t count;
    void (*fn)(void *, size_t);
    void *ctx;
    std::atomic<size_t> next{0};     // next index to hand out
    std::atomic<size_t> done{0};     // indices finished
    int refs = 0;                    // workers inside the job (under Pool::m)
};

thread_local bool t_pool_worker = false;

void run_indices(Job *j)
{
    for (size_t i; (i = j->next.fetch_add(1)) < j->count;) {
        j->fn(j->ctx, i);
        j->done.fetch_add(1);
    }
}

class Pool {
public:
    explicit Pool(int workers)
    {
        // a thread that cannot be started leaves fewer workers (callers finish alone)
        try {
            for (int w = 0; w < workers; ++w) std::thread([this] { work(); }).detach();
        } catch (...) {
        }
    }

    void run(Job *j)
    {
        {
            std::lock_guard<std::mutex> lk(m_);
            q_.push_back(j);
        }
        cv_.notify_all();
        run_indices(j);
        std::unique_lock<std::mutex> lk(m_);
        for (auto it = q_.begin(); it != q_.end(); ++it)
            if (*it == j) {
                q_.erase(it);
                break;
            }
        done_.wait(lk, [&] { return j->refs == 0 && j->done.load() == j->count; });
    }

private:
    void work()
    {
        t_pool_worker = true;
        std::unique_lock<std::mutex> lk(m_);
        for (;;) {
            cv_.wait(lk, [&] { return !q_.empty(); });
            Job *j = q_.front();
            ++j->refs;
            lk.unlock();
            run_indices(j);
            lk.lock();
            // no index left: take the job off the queue so that idle workers sleep
            if (!q_.empty() && q_.front() == j) q_.pop_front();
            if (--j->refs == 0) done_.notify_all();
        }
    }

    std::mutex m_;
    std::condition_variable cv_, done_;
    std::deque<Job *> q_;
};

// fixed at the first call, so the serial check below and the pool's size
// always agree (and the planners' hot loops make no system call for it)
int pool_threads()
{
    static const int t = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 16u);
    return t;
}

Pool *pool()
{
    static Pool *p = new Pool(pool_threads() - 1);
    return p;
}

}  // namespace

void parallel_run(size_t count, void (*fn)(void *, size_t), void *ctx)
{
    if (count <= 1 || t_pool_worker || pool_threads() <= 1) {
        for (size_t i = 0; i < count; ++i) fn(ctx, i);
        return;
    }
    Job j;
    j.count = count;
    j.fn = fn;
    j.ctx = ctx;
    pool()->run(&j);
}

}  // namespace qsim
