// cm_profile.cu -- tracing: per-kernel CUDA-event timing and launch counting.
//
// When enabled, every kernel the library launches is bracketed by two CUDA
// events recorded on its own launch stream; cm_profile_collect() waits for
// them and sums the elapsed times per kernel name.  The launch counter counts
// every kernel the library enqueues (also when profiling is off).  Events come
// from a pool and are reused, so profiling adds two event records per launch
// and no allocation after warm-up.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/cm.h"
#include "cm_launch.h"

namespace cmk {

namespace {

struct Pending {
    const char* name;
    cudaEvent_t a, b;
};

struct Stat {
    std::string name;
    long long launches;
    double ms;
};

std::mutex g_mu;
bool g_on = false;
std::vector<cudaEvent_t> g_pool;
std::vector<Pending> g_pending;
std::vector<Stat> g_stats;
long long g_launches = 0;

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

}  // namespace

KernelScope::KernelScope(const char* name, cudaStream_t s, int launches) : name_(name), s_(s), a_(nullptr)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!capturing(s)) g_launches += launches;
    if (g_on && !capturing(s)) {
        a_ = take_event();
        if (a_) cudaEventRecord(a_, s);
    }
}

KernelScope::~KernelScope()
{
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = take_event();
    if (!b) {
        g_pool.push_back(a_);
        return;
    }
    cudaEventRecord(b, s_);
    g_pending.push_back({name_, a_, b});
}

void count_launches(long long n)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_launches += n;
}

bool profiling_on()
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_on;
}

cudaEvent_t profile_take_event()
{
    std::lock_guard<std::mutex> lk(g_mu);
    return take_event();
}

void profile_push(const char* name, cudaEvent_t a, cudaEvent_t b)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back({name, a, b});
}

}  // namespace cmk

using namespace cmk;

extern "C" {

int cm_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    return CM_OK;
}

int cm_profile_collect(cm_kernel_stat* out, int32_t cap, int32_t* count)
{
    std::lock_guard<std::mutex> lk(g_mu);
    int st = CM_OK;
    for (const Pending& p : g_pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) {
            st = CM_ECUDA;
        } else {
            bool found = false;
            for (Stat& s : g_stats) {
                if (s.name == p.name) {
                    s.launches += 1;
                    s.ms += ms;
                    found = true;
                    break;
                }
            }
            if (!found) g_stats.push_back({p.name, 1, (double)ms});
        }
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
    const int n = (int)g_stats.size();
    if (count) *count = n;
    if (out) {
        for (int i = 0; i < n && i < cap; ++i) {
            std::memset(out[i].name, 0, sizeof(out[i].name));
            std::strncpy(out[i].name, g_stats[i].name.c_str(), sizeof(out[i].name) - 1);
            out[i].launches = g_stats[i].launches;
            out[i].total_ms = g_stats[i].ms;
        }
    }
    return st;
}

int cm_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (const Pending& p : g_pending) {
        cudaEventSynchronize(p.b);
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
    g_stats.clear();
    return CM_OK;
}

int64_t cm_launch_count(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_launches;
}

}  // extern "C"
