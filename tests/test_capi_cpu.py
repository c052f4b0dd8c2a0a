"""CPU-side checks of the C-ABI library: it loads, exports every entry point
declared in include/dzs.h, and its host-only calls work without a GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dzs():
    from paper_2005_05328_gb300 import build
    build.build()
    import paper_2005_05328_gb300 as m
    m.load()
    return m


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dzs.h")).read()
    return sorted(set(re.findall(r"^DZS_API\s+[\w\s\*]+?\b(dzs_\w+)\s*\(", src, flags=re.M)))


def test_header_and_binding_agree():
    import paper_2005_05328_gb300 as m
    assert declared_functions() == sorted(m.EXPORTED)


def test_library_exports_every_declared_symbol(dzs):
    lib = dzs.load()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_params_default_roundtrip(dzs):
    p = dzs.params()
    assert (p.n1d, p.mesh, p.box, p.nsteps) == (32, 64, 64.0, 96)
    assert (p.leaf_bucket, p.walk_group, p.merge_level) == (8, 32, 2)
    assert p.theta == 0.5 and p.theta_dzs == 0.1 and p.rs_cells == 1.25 and p.rcut_rs == 4.5
    assert p.soft_frac == 1 / 40 and p.buffer_cells == 2.0 and p.seed == 1 and p.lc_capacity == 0


def test_footprint_and_validation(dzs):
    small = dzs.dzs_footprint_bytes(dzs.params())
    big = dzs.dzs_footprint_bytes(dzs.params(n1d=128, mesh=256, box=256.0, merge_level=3))
    assert 0 < small < big
    # ~ a few hundred bytes per particle plus the mesh
    assert big < 2000 * 128 ** 3
    with pytest.raises(dzs.DzsError) as e:
        dzs.dzs_footprint_bytes(dzs.params(mesh=100))
    assert e.value.status == dzs.DZS_EINVAL
    with pytest.raises(dzs.DzsError):
        dzs.dzs_footprint_bytes(dzs.params(leaf_bucket=40))


def test_create_without_gpu_fails_cleanly(dzs):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dzs.DzsError) as e:
        dzs.dzs_create(dzs.params())
    assert e.value.status == dzs.DZS_EDEVICE


def test_capacity_shrinks_footprint(dzs):
    """a context re-created after a halt with fewer particle slots holds less
    device memory; capacity above n1d^3 is rejected"""
    kw = dict(n1d=128, mesh=256, box=256.0, merge_level=3)
    full = dzs.dzs_footprint_bytes(dzs.params(**kw))
    small = dzs.dzs_footprint_bytes(dzs.params(capacity=128 ** 3 // 16, **kw))
    assert small < full - 0.9 * (full - dzs.dzs_footprint_bytes(dzs.params(capacity=1, **kw)))
    with pytest.raises(dzs.DzsError) as e:
        dzs.dzs_footprint_bytes(dzs.params(capacity=128 ** 3 + 1, **kw))
    assert e.value.status == dzs.DZS_EINVAL
    p = dzs.params()
    assert p.capacity == 0 and p.dzs_criterion == dzs.CRIT_GEOMETRIC and p.alpha_dyn == 0.01


def test_struct_layouts_match_the_header(tmp_path, dzs):
    """sizeof / offsetof of the C structs equal the ctypes mirrors"""
    import ctypes
    import subprocess
    fields = [f[0] for f in dzs.Params._fields_]
    halt = [f[0] for f in dzs.Halt._fields_]
    body = ["#include <stdio.h>", "#include <stddef.h>", '#include "dzs.h"', "int main(void) {",
            '  printf("%zu\\n", sizeof(dzs_params));']
    body += ['  printf("%%zu\\n", offsetof(dzs_params, %s));' % f for f in fields]
    body += ['  printf("%zu\\n", sizeof(dzs_halt));']
    body += ['  printf("%%zu\\n", offsetof(dzs_halt, %s));' % f for f in halt]
    obs = [f[0] for f in dzs.Observe._fields_]
    body += ['  printf("%zu\\n", sizeof(dzs_observe));']
    body += ['  printf("%%zu\\n", offsetof(dzs_observe, %s));' % f for f in obs]
    extra = [("dzs_request", dzs.Request), ("dzs_request_result", dzs.RequestResult),
             ("dzs_serve_config", dzs.ServeConfig)]
    body += ['  printf("%zu\\n", sizeof(dzs_halo));']
    body += ['  printf("%%zu\\n", offsetof(dzs_halo, %s));' % f for f in dzs.HALO_DTYPE.names]
    for cname, cls in extra:
        body += ['  printf("%%zu\\n", sizeof(%s));' % cname]
        body += ['  printf("%%zu\\n", offsetof(%s, %s));' % (cname, f[0]) for f in cls._fields_]
    body += ['  printf("%zu\\n", sizeof(dzs_lc_record));', "  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(body) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(dzs.Params)] + [getattr(dzs.Params, f).offset for f in fields]
    want += [ctypes.sizeof(dzs.Halt)] + [getattr(dzs.Halt, f).offset for f in halt]
    want += [ctypes.sizeof(dzs.Observe)] + [getattr(dzs.Observe, f).offset for f in obs]
    want += [dzs.HALO_DTYPE.itemsize] + [dzs.HALO_DTYPE.fields[f][1] for f in dzs.HALO_DTYPE.names]
    for cname, cls in extra:
        want += [ctypes.sizeof(cls)] + [getattr(cls, f[0]).offset for f in cls._fields_]
    want += [dzs.RECORD_DTYPE.itemsize]
    assert got == want


def test_noalloc_sort_source_allocates_nothing():
    """the allocation-free sort's entry point calls no allocating CUDA routine"""
    import re
    src = open(os.path.join(ROOT, "paper_2005_05328_gb300", "csrc", "sort.cu")).read()
    body = src[src.index('extern "C" dzs_status dzs_morton_sort_noalloc'):]
    body = body[:body.index("\n}\n") + 3]
    assert not re.search(r"cudaMalloc|cudaFree|cudaMallocAsync|cudaHostAlloc|new |malloc\(", body)


def test_autotune_cache_path_follows_the_environment(monkeypatch, tmp_path):
    from paper_2005_05328_gb300 import autotune
    monkeypatch.setenv("DZS_TUNE_CACHE", str(tmp_path / "x.json"))
    assert autotune.cache_path() == str(tmp_path / "x.json")
    assert autotune._load() == {}
    autotune._store({"k": {"walk_eval": 1}})
    assert autotune._load() == {"k": {"walk_eval": 1}}
