"""Host-side checks of the C ABI: the library loads, exports what include/pbs.h declares,
and its host-only entry points behave (no GPU needed)."""
import ctypes as ct
import subprocess

import pytest

import paper_2304_00337_gb300 as pbs


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as ge
    ge.build()
    return pbs.lib()


def test_exports_every_declared_symbol(built):
    declared = pbs.abi_symbols_from_header()
    assert len(declared) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", pbs.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(built, s)


def test_default_opts_and_strerror(built):
    o = pbs.default_opts()
    assert (o.nev, o.block, o.span, o.precision, o.coarsest, o.nodal_cycles, o.extrap_depth) == (4, 6, 3, 1, 4, 2, 3)
    assert o.tol == 1e-8 and o.max_iter == 400 and o.kbatch == 1
    assert pbs.strerror(pbs.PBS_EINVAL) == "invalid argument"
    assert pbs.strerror(12345) == "unknown status"


def test_num_levels_rule(built):
    assert pbs.num_levels(256, 256, 4) == 7
    assert pbs.num_levels(48, 32, 4) == 4
    assert pbs.num_levels(6, 6, 4) == 1
    assert pbs.num_levels(1, 6, 4) == pbs.PBS_EINVAL


def test_null_arguments_are_rejected(built):
    L = built
    assert L.pbs_create(None, 0, 0) == pbs.PBS_EINVAL
    assert L.pbs_destroy(None) == pbs.PBS_OK
    assert L.pbs_solve_k(None, None, None, None, None, None, None, None, None) == pbs.PBS_EINVAL
    assert L.pbs_apply(None, None, None, 0, 0, None, 1, None, None, None) == pbs.PBS_EINVAL
    assert L.pbs_m_householder(None, None, None, 4, None, None, None, None) == pbs.PBS_EINVAL


def test_struct_layout_matches_header(built):
    # pbs_opts: 5 ints, 2 doubles, 5 ints, 1 uint64, 1 int with natural alignment
    assert ct.sizeof(pbs.pbs_opts) == 80
    assert ct.sizeof(pbs.pbs_geom) == 32


def test_job_bytes_admission_estimate(built):
    # pbs_job_bytes is host arithmetic: the device bytes a path job needs
    o = dict(nev=8, block=10, kbatch=4)
    b256 = pbs.job_bytes(256, 256, o, 31)
    assert 1e8 < b256 < 2e10
    assert pbs.job_bytes(256, 256, dict(o, kbatch=8), 31) > b256  # more Bloch vectors in flight
    assert pbs.job_bytes(512, 512, o, 31) > 3 * b256  # four times the unknowns
    # a chain needs extrapolation history; all Bloch vectors in flight need none
    assert pbs.job_bytes(256, 256, dict(o, kbatch=31), 31) < pbs.job_bytes(256, 256, dict(o, kbatch=31), 62)
    # 1024 x 1024, 64 Bloch vectors in flight, block 10, fits one 288 GB device
    # (multigrid work is chunked to a fixed byte size, so both policies need about the same)
    c3 = pbs.job_bytes(1024, 1024, dict(nev=8, block=10, kbatch=64), 64)
    assert 64 * 40 * 32 * 2 ** 20 < c3 < 250e9  # at least the four role blocks of 640 FP64 columns
    assert pbs.job_bytes(1024, 1024, dict(nev=8, block=10, kbatch=64, precision=pbs.PBS_FP64), 64) < 250e9
    with pytest.raises(pbs.PbsError) as e:
        pbs.job_bytes(255, 256, o, 4)
    assert e.value.status == pbs.PBS_EINVAL
