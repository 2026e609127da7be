"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/mpmcr.h declares; argument validation that happens before
any device work is checked here too (no compute calls without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpmcr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mpm_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_05046_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mpm_create", "mpm_add_particles", "mpm_set_rigid_bodies", "mpm_step",
                     "mpm_get_particles", "mpm_get_rigid_impulses", "mpm_destroy",
                     "mpm_tape_begin", "mpm_tape_end", "mpm_backward", "mpm_contact_adjoint",
                     "mpm_set_rigid_dynamics", "mpm_set_material"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), "libmpmcr.so does not export %s" % name


def test_binding_covers_every_symbol():
    from paper_2503_05046_gb300 import native
    assert set(declared_functions()) <= set(native.SIGNATURES)


def test_argument_validation_without_device(lib):
    from paper_2503_05046_gb300 import native
    out = C.c_void_p()
    spec = native.GridSpec()
    spec.dx = 0.01
    spec.res[0], spec.res[1], spec.res[2] = 30, 32, 32  # not a multiple of 4
    spec.max_particles = 10
    spec.max_contacts = 10
    assert native.lib.mpm_create(C.byref(spec), None, C.byref(out)) == native.ERR_INVALID_ARG
    spec.res[0] = 32
    spec.dx = -1.0
    assert native.lib.mpm_create(C.byref(spec), None, C.byref(out)) == native.ERR_INVALID_ARG
    assert native.lib.mpm_create(None, None, C.byref(out)) == native.ERR_INVALID_ARG
    spec.dx = 0.01
    spec.max_blocks = -1  # block-sparse pool
    assert native.lib.mpm_create(C.byref(spec), None, C.byref(out)) == native.ERR_INVALID_ARG
    spec.max_blocks = 0
    spec.res[0], spec.res[1], spec.res[2] = 2048, 2048, 1024  # 2^32 nodes: ids overflow 32 bits
    assert native.lib.mpm_create(C.byref(spec), None, C.byref(out)) == native.ERR_INVALID_ARG
    assert native.lib.mpm_num_particles(None, None) == native.ERR_INVALID_ARG
    assert native.lib.mpm_step(None, 1e-4, 1, None, None) == native.ERR_INVALID_ARG
    assert native.lib.mpm_set_rigid_dynamics(None, 0, None) == native.ERR_INVALID_ARG
    assert native.lib.mpm_set_option(None, native.OPT_GRAPHS, 1) == native.ERR_INVALID_ARG
    assert native.lib.mpm_contact_adjoint(None, native.MEM_HOST, 0, None, None, None, 0, None,
                                          None, None, None) == native.ERR_INVALID_ARG
    assert native.lib.mpm_tape_begin(None) == native.ERR_INVALID_ARG
    assert native.lib.mpm_tape_end(None) == native.ERR_INVALID_ARG
    assert native.lib.mpm_backward(None, native.MEM_HOST, None, None, None, None, None, None,
                                   None, None, None, None, None, None, None) == native.ERR_INVALID_ARG
    assert native.lib.mpm_set_material(None, 0, None) == native.ERR_INVALID_ARG
    assert native.lib.mpm_add_cloth(None, 3, None, None, 1, None, 1e-3, None, native.MEM_HOST,
                                    None) == native.ERR_INVALID_ARG
    assert native.lib.mpm_set_pins(None, 0, None, None) == native.ERR_INVALID_ARG
    assert native.lib.mpm_destroy(None) == native.OK
    assert native.lib.mpm_last_error(None) == b"invalid mpm context"
    # batches: bad handles and member lists are refused before any device work
    assert native.lib.mpm_batch_create(None, 1, C.byref(out)) == native.ERR_INVALID_ARG
    members = (C.c_void_p * 2)(None, None)
    assert native.lib.mpm_batch_create(members, 2, C.byref(out)) == native.ERR_INVALID_ARG
    assert native.lib.mpm_batch_create(members, 0, C.byref(out)) == native.ERR_INVALID_ARG
    assert native.lib.mpm_batch_step(None, 1e-4, 1, None) == native.ERR_INVALID_ARG
    assert native.lib.mpm_batch_sort(None) == native.ERR_INVALID_ARG
    assert native.lib.mpm_batch_synchronize(None, None, None) == native.ERR_INVALID_ARG
    assert native.lib.mpm_batch_set_option(None, native.BATCH_OPT_GRAPHS, 1) == native.ERR_INVALID_ARG
    assert native.lib.mpm_batch_last_error(None) == b"invalid mpm batch"
    native.lib.mpm_batch_destroy(None)


def test_oracle_is_separate_from_the_cuda_library():
    """The oracle shares no source with the CUDA path and neither includes the
    other's headers."""
    csrc = os.path.join(ROOT, "paper_2503_05046_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "mpm_oracle" not in text and "orc_" not in text
    otext = open(os.path.join(ROOT, "oracle", "mpm_oracle.c")).read()
    assert "mpmcr.h" not in otext and "common.cuh" not in otext
    for f in os.listdir(os.path.join(ROOT, "paper_2503_05046_gb300")):
        if f.endswith(".py"):
            text = open(os.path.join(ROOT, "paper_2503_05046_gb300", f)).read()
            assert "import oracle" not in text and "from oracle" not in text
