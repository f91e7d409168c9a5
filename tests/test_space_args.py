"""Argument checks of bo_space_create through the C ABI, on the CPU.

Every check of the descriptor runs before the library touches a device, so a
bad descriptor is refused with BO_ERR_ARG and a message naming the field on a
machine without a GPU too.  (The values that the checks accept are exercised
by every GPU test that creates a space.)
"""
import ctypes as C

import numpy as np
import pytest

BO_ERR_ARG = 1


@pytest.fixture(scope="module")
def lib():
    from paper_2111_14991_gb300 import bo, build
    build.build()
    return bo.lib()


def create(lib, grids, invalid=None, **kw):
    from paper_2111_14991_gb300 import bo
    desc, keep = bo.make_desc(grids, invalid, **kw)
    out = C.c_void_p()
    rc = lib.bo_space_create(C.byref(desc), C.byref(out))
    msg = lib.bo_last_error().decode()
    del keep
    return rc, msg, desc


GRIDS = [np.linspace(0.0, 1.0, 4), np.linspace(0.0, 1.0, 3)]


@pytest.mark.parametrize("field, value, words", [
    ("nu", 0.5, "nu"),
    ("lengthscale", 0.0, "lengthscale"),
    ("lengthscale", float("nan"), "lengthscale"),
    ("jitter", -1e-12, "jitter"),
    ("af", 7, "af"),
    ("explore", 5, "explore"),
    ("precision", 9, "precision"),
    ("n_max", 0, "n_max"),
    ("n_max", 513, "n_max"),
    ("skip_threshold", -1, "negative"),
    ("n_init", -2, "negative"),
    ("init_designs", -3, "negative"),
    ("init_mode", 4, "init_mode"),
])
def test_bad_descriptor_field(lib, field, value, words):
    from paper_2111_14991_gb300 import bo
    desc, keep = bo.make_desc(GRIDS)
    setattr(desc, field, value)
    out = C.c_void_p()
    rc = lib.bo_space_create(C.byref(desc), C.byref(out))
    assert rc == BO_ERR_ARG and out.value is None
    assert words in lib.bo_last_error().decode()


def test_parameter_count(lib):
    rc, msg, _ = create(lib, [])
    assert rc == BO_ERR_ARG and "d = 0" in msg
    rc, msg, _ = create(lib, [np.array([0.0, 1.0])] * 17)
    assert rc == BO_ERR_ARG and "d = 17" in msg


@pytest.mark.parametrize("grid, words", [
    (np.array([]), "bad value list"),
    (np.linspace(0.0, 1.0, 257), "bad value list"),
    (np.array([0.0, 1.5]), "not normalized"),
    (np.array([-0.25, 0.5]), "not normalized"),
    (np.array([0.0, np.nan]), "not normalized"),
])
def test_bad_value_list(lib, grid, words):
    rc, msg, _ = create(lib, [np.linspace(0.0, 1.0, 3), grid])
    assert rc == BO_ERR_ARG and words in msg and "parameter 1" in msg


def test_space_too_large(lib):
    rc, msg, _ = create(lib, [np.linspace(0.0, 1.0, 256)] * 6)   # 2^48 configurations
    assert rc == BO_ERR_ARG and "too large" in msg


def test_no_valid_configuration(lib):
    invalid = np.ones(4 * 3, dtype=np.uint8)
    rc, msg, _ = create(lib, GRIDS, invalid)
    assert rc == BO_ERR_ARG and "no valid configuration" in msg


def test_null_arguments(lib):
    out = C.c_void_p()
    assert lib.bo_space_create(None, C.byref(out)) == BO_ERR_ARG
    from paper_2111_14991_gb300 import bo
    desc, keep = bo.make_desc(GRIDS)
    assert lib.bo_space_create(C.byref(desc), None) == BO_ERR_ARG
    desc.values = None
    assert lib.bo_space_create(C.byref(desc), C.byref(out)) == BO_ERR_ARG
    assert "missing" in lib.bo_last_error().decode()


def test_server_open_checks_the_descriptor(lib):
    """bo_server_open refuses a bad descriptor at once, with the same checks and
    messages as bo_space_create, and registers nothing; a good one is queued.
    (The server's worker only waits here: nothing is admitted without a device
    budget, so this runs without a GPU.)"""
    from paper_2111_14991_gb300 import bo
    cfg = bo.ServerConfig()
    cfg.budget_bytes = 1          # below any session: a good descriptor gets BO_ERR_NOMEM, not BO_ERR_ARG
    cfg.max_sessions = 4
    srv = C.c_void_p()
    assert lib.bo_server_create(C.byref(cfg), C.byref(srv)) == 0
    try:
        sid = C.c_int64(-1)
        for field, value, words in (("nu", 0.5, "nu"), ("precision", 9, "precision"), ("n_max", 0, "n_max"),
                                    ("lengthscale", -1.0, "lengthscale")):
            desc, keep = bo.make_desc(GRIDS)
            setattr(desc, field, value)
            assert lib.bo_server_open(srv, C.byref(desc), C.byref(sid)) == BO_ERR_ARG
            assert words in lib.bo_last_error().decode()
        desc, keep = bo.make_desc([np.linspace(0.0, 1.0, 3), np.array([0.0, 2.0])])
        assert lib.bo_server_open(srv, C.byref(desc), C.byref(sid)) == BO_ERR_ARG
        assert "not normalized" in lib.bo_last_error().decode()
        desc, keep = bo.make_desc(GRIDS, np.ones(12, dtype=np.uint8))
        assert lib.bo_server_open(srv, C.byref(desc), C.byref(sid)) == BO_ERR_ARG
        assert "no valid configuration" in lib.bo_last_error().decode()
        desc, keep = bo.make_desc(GRIDS)
        assert lib.bo_server_open(srv, C.byref(desc), C.byref(sid)) == 6     # BO_ERR_NOMEM: over the budget
        st = bo.ServerStats()
        assert lib.bo_server_stats_get(srv, C.byref(st)) == 0
        assert st.queued == 0 and st.admitted == 0
    finally:
        assert lib.bo_server_destroy(srv) == 0
