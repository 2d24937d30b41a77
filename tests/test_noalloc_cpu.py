"""Host-side parts of dbt_integrate_scan_noalloc, checked without a GPU.

Callers that cannot allocate device memory while they run use the
library's fixed scratch array through dbt_integrate_scan_noalloc.  Its size
limits are checked on the host before any CUDA call (dbt_noalloc_check
exposes the same check), and the array's device address is remembered per
CUDA context (csrc/scratch_cache.h), so that a context created later on the
same device never receives an address that belonged to an earlier one.
"""
import os
import subprocess

import pytest

import paper_2509_20081_gb300 as dbt
from paper_2509_20081_gb300 import dbtsdf as B

CSRC = os.path.join(os.path.dirname(B.__file__), "csrc")


def test_limits_on_the_host():
    dbt.lib()
    B.dbt_noalloc_check(1600, 1600, 320, 11, 65536)         # the urban grid at the limit
    B.dbt_noalloc_check(128, 128, 128, 21, 0)
    with pytest.raises(dbt.DbtError) as e:
        B.dbt_noalloc_check(64, 64, 64, 11, 65537)
    assert e.value.status == B.DBT_EINVAL and "65536" in str(e.value)
    with pytest.raises(dbt.DbtError) as e:                  # 4.2 M bricks
        B.dbt_noalloc_check(4096, 4096, 512, 11, 10)
    assert e.value.status == B.DBT_EINVAL and "too large" in str(e.value)
    with pytest.raises(dbt.DbtError):                       # 520,192 bricks: fit at K = 11 only
        B.dbt_noalloc_check(2048, 2032, 256, 21, 65536)
    B.dbt_noalloc_check(2048, 2032, 256, 11, 65536)
    for bad in ((64, 64, 64, 10, 5), (64, 64, 64, 23, 5), (0, 64, 64, 11, 5), (64, 64, 64, 11, -1)):
        with pytest.raises(dbt.DbtError):
            B.dbt_noalloc_check(*bad)


_CACHE_TEST = r"""
#include <cstdio>
#include "scratch_cache.h"
#define CHECK(c) do { if (!(c)) { std::printf("FAIL line %d\n", __LINE__); return 1; } } while (0)
int main() {
    ContextAddressCache<4> c;
    int a, b, x;
    CHECK(c.find(7) == nullptr);
    c.put(7, &a);
    CHECK(c.find(7) == &a);
    // a context created later (new id, e.g. after a device reset) misses and gets its own lookup
    CHECK(c.find(8) == nullptr);
    c.put(8, &b);
    CHECK(c.find(8) == &b && c.find(7) == &a);
    c.put(7, &x);                                   // same context again: replaced, not duplicated
    CHECK(c.find(7) == &x);
    for (unsigned long long id = 100; id < 104; ++id) c.put(id, &a);
    CHECK(c.find(7) == nullptr && c.find(8) == nullptr);   // evicted, never stale
    CHECK(c.find(100) == &a && c.find(103) == &a);
    std::printf("OK\n");
    return 0;
}
"""


def test_scratch_address_cache_is_per_context(tmp_path):
    src = tmp_path / "t.cc"
    exe = tmp_path / "t"
    src.write_text(_CACHE_TEST)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout
