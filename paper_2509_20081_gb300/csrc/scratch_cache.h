// Device addresses of one __device__ array, remembered per CUDA context.
//
// A __device__ array has a separate instance, at its own address, in every
// context that loads the module: a context created later on the same device
// (after cudaDeviceReset, or a second driver context) gets a new instance.
// Entries are keyed by the context's unique id (cuCtxGetId: unique for the
// life of the process), so an address taken in a context that no longer
// exists is never handed out for a new one.  Plain C++ without CUDA headers,
// so that its logic is tested on a machine without a GPU; callers lock.
#pragma once

template <int N>
struct ContextAddressCache {
    struct Entry {
        unsigned long long ctx_id;
        void *addr;               // null: empty slot
    };
    Entry e[N] = {};
    int next = 0;                 // slot replaced when every slot is in use

    void *find(unsigned long long ctx_id) const {
        for (int i = 0; i < N; ++i)
            if (e[i].addr && e[i].ctx_id == ctx_id) return e[i].addr;
        return nullptr;
    }

    void put(unsigned long long ctx_id, void *addr) {
        for (int i = 0; i < N; ++i)
            if (e[i].addr && e[i].ctx_id == ctx_id) {
                e[i].addr = addr;
                return;
            }
        e[next] = Entry{ctx_id, addr};
        next = (next + 1) % N;
    }
};
