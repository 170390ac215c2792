"""The C ABI without a GPU: the library builds, loads, exports every entry
point include/boruta.h declares, and rejects bad arguments on the host."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_09950_gb300 import boruta, build

    build.build()
    return boruta.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "boruta.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(boruta_\w+)\s*\(", text)))


def test_header_and_binding_agree():
    from paper_2605_09950_gb300 import boruta

    assert declared_functions() == sorted(boruta.EXPORTS)


def _struct_fields(name):
    text = open(os.path.join(ROOT, "include", "boruta.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", text).group(1)
    return [re.findall(r"(\w+)(?:\[\w*\])?\s*$", decl.strip())[0]
            for stmt in body.split(";") if stmt.strip() for decl in stmt.split(",")
            if re.findall(r"(\w+)(?:\[\w*\])?\s*$", decl.strip())]


@pytest.mark.parametrize("cname,pyname", [("boruta_opts", "Opts"), ("boruta_result", "Result"),
                                          ("boruta_job", "Job")])
def test_binding_structs_follow_the_header(cname, pyname):
    """The ctypes structures list the header's fields in the header's order."""
    from paper_2605_09950_gb300 import boruta

    assert [f for f, _ in getattr(boruta, pyname)._fields_] == _struct_fields(cname)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_default_opts(lib):
    from paper_2605_09950_gb300 import boruta

    o = boruta.Opts()
    lib.boruta_default_opts(o)
    assert o.kl_eps == 1e-7 and o.precision == 0 and o.tie_break == 0 and o.stat == 0


@pytest.mark.parametrize("bad", [
    dict(N=0), dict(N=1 << 24), dict(n_bins=1), dict(n_bins=257), dict(max_iter=0), dict(max_iter=127),
    dict(max_depth=31), dict(n_trees=0), dict(alpha=0.0), dict(task=4), dict(mtry=-1),
    dict(n_classes=9), dict(precision=2), dict(band_launch=3), dict(band_launch=-1), dict(autotune=2),
])
def test_invalid_arguments_are_rejected_on_the_host(lib, bad):
    from paper_2605_09950_gb300 import boruta

    X = np.zeros((3, 16), np.uint8)
    y = np.zeros(16, np.uint8)
    args = dict(task=0, n_trees=2, max_depth=3, mtry=0, n_bins=4, max_iter=3, alpha=0.01, seed=0, N=16)
    opts = dict(host_inputs=1)
    for k, v in bad.items():
        (opts if k in ("n_classes", "precision", "band_launch", "autotune") else args)[k] = v
    with pytest.raises(boruta.BorutaError) as e:
        boruta.boruta_fit(X, y, **args, **opts)
    assert e.value.code == -1
    assert str(e.value)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2605_09950_gb300 import boruta

    monkeypatch.setattr(boruta, "_lib", None)
    monkeypatch.setattr(boruta, "_LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="missing"):
        boruta.lib()


def test_quantise_and_batch_reject_bad_arguments_on_the_host(lib):
    """Argument checks run before any CUDA call (no GPU needed)."""
    import ctypes as ct

    from paper_2605_09950_gb300 import boruta

    L = boruta.lib()
    # quantise: NULL pointers, N < 1, ld < N, bins outside [2, 256]
    assert L.boruta_quantise(None, 16, 16, 2, 8, None, 16, None) == -1
    buf = (ct.c_float * 32)()
    out = (ct.c_uint8 * 32)()
    assert L.boruta_quantise(ct.addressof(buf), 16, 0, 2, 8, ct.addressof(out), 16, None) == -1
    assert L.boruta_quantise(ct.addressof(buf), 8, 16, 2, 8, ct.addressof(out), 16, None) == -1
    assert L.boruta_quantise(ct.addressof(buf), 16, 16, 2, 1, ct.addressof(out), 16, None) == -1
    assert L.boruta_quantise(ct.addressof(buf), 16, 16, 2, 257, ct.addressof(out), 16, None) == -1
    assert b"n_bins" in L.boruta_last_error()
    # batch: negative job count, NULL output handle, NULL batch
    h = ct.c_void_p()
    assert L.boruta_batch_create(-1, None, None, ct.byref(h)) == -1
    assert L.boruta_batch_create(0, None, None, None) == -1
    running = ct.c_int32()
    assert L.boruta_batch_step(None, ct.byref(running)) == -1
    assert L.boruta_batch_run(None, 1, ct.byref(running)) == -1
    assert L.boruta_batch_read(None, 0, None, None, None, None, None) == -1
    L.boruta_batch_destroy(None)


def test_rank_and_median_selection_match_the_oracle(lib):
    """The library's host-side ranking and median selection (no GPU) equal
    the oracle's on random finished runs with NaN gaps and ties."""
    import oracle
    from paper_2605_09950_gb300 import boruta

    rng = np.random.default_rng(11)
    for trial in range(30):
        T, p = int(rng.integers(1, 15)), int(rng.integers(1, 30))
        runs = []
        for r in range(int(rng.integers(1, 8))):
            it = int(rng.integers(1, T + 1))
            h = np.full((T, p), np.nan)
            h[:it] = np.round(rng.random((it, p)) * 4) / 4  # coarse values: ties
            h[1:it][rng.random((it - 1, p)) < 0.3] = np.nan
            sm = np.full(T, np.nan)
            sm[:it] = np.round(rng.random(it) * 4) / 4
            dec = rng.integers(-1, 2, size=p).astype(np.int8)
            runs.append(dict(imp_history=h, shadow_max=sm, iterations=it, decision=dec))
            np.testing.assert_array_equal(boruta.boruta_rank(dec, h, it), oracle.rank(dec, h, it))
        got = boruta.boruta_select_median(runs)
        want = oracle.select_median(runs)
        np.testing.assert_array_equal(got[0], want[0])
        assert got[1] == want[1]
        np.testing.assert_array_equal(got[2], want[2])
