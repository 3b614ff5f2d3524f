"""C-ABI checks that need no GPU: the library builds and loads, exports every
entry point include/mtgp.h declares, and its host-only parameter-set code
agrees with the oracle (parity of the parameter-load step)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1501_07701_gb300 import build as mbuild
from paper_1501_07701_gb300 import mtgp, workloads
from tests.conftest import ROOT, read_golden


@pytest.fixture(scope="module")
def lib():
    mbuild.build()
    return mtgp.load_library()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mtgp_\w+)\s*\(", src, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    assert _declared_functions() <= set(mtgp._SIGS)


def test_version(lib):
    assert "sm_103a" in mtgp.mtgp_version()


@pytest.mark.parametrize("mexp", [3217, 4253, 9689, 11213, 19937, 21701, 23209, 44497, 80, 70])
@pytest.mark.parametrize("seed", [0x5EED, 0, 12345])
def test_params_generate_matches_oracle(lib, mexp, seed):
    p = mtgp.mtgp_params_generate(mexp, seed)
    d = mtgp.mtgp_params_get(p)
    o = oracle.params_generate(mexp, seed)
    assert (d["mexp"], d["n"], d["pos"], d["sh1"], d["sh2"], d["mask"]) == \
        (o.mexp, o.n, o.pos, o.sh1, o.sh2, o.mask)
    assert d["rec_tbl"] == list(o.rec_tbl)
    assert d["tmp_tbl"] == list(o.tmp_tbl)


def test_params_load_basis_and_tables(lib, golden_dir, tmp_path):
    g = read_golden(os.path.join(golden_dir, "hand_example_n3.txt"))
    p = mtgp.mtgp_params_load(os.path.join(golden_dir, "hand_example_n3.txt"))
    d = mtgp.mtgp_params_get(p)
    assert d["n"] == 3 and d["mask"] == 0xFFFF0000 and d["pos"] == 2
    assert d["rec_tbl"][0xF] == 0xF0000000 and d["tmp_tbl"][12] == 12
    # the same set written as full tables
    f = tmp_path / "p.txt"
    f.write_text("mexp 80\npos 2 # comment\nsh1 1\nsh2 2\nrec_tbl %s\ntmp_tbl %s\n" % (
        " ".join(hex(v) for v in d["rec_tbl"]), " ".join(str(v) for v in d["tmp_tbl"])))
    d2 = mtgp.mtgp_params_get(mtgp.mtgp_params_load(str(f)))
    assert d2 == d
    assert g["mexp"] == [80]


@pytest.mark.parametrize("text,status", [
    ("mexp 80\npos 2\nsh1 1\nsh2 2\nrec_basis 1 2 4 8\n", 6),              # missing tmp
    ("mexp 80\npos 3\nsh1 1\nsh2 2\nrec_basis 1 2 4 8\ntmp_basis 1 2 4 8\n", 1),   # pos >= N
    ("mexp 80\npos 2\nsh1 32\nsh2 2\nrec_basis 1 2 4 8\ntmp_basis 1 2 4 8\n", 1),  # shift
    ("mexp 96\npos 2\nsh1 1\nsh2 2\nrec_basis 1 2 4 8\ntmp_basis 1 2 4 8\n", 1),   # r = 32
    ("mexp 80\npos 2\nsh1 1\nsh2 2\nrec_tbl " + " ".join(["1"] * 16) +
     "\ntmp_basis 1 2 4 8\n", 1),                                                # non-linear
    ("mexp 80\npos zz\n", 6),
])
def test_params_load_rejects(lib, tmp_path, text, status):
    f = tmp_path / "bad.txt"
    f.write_text(text)
    with pytest.raises(mtgp.MtgpError) as ei:
        mtgp.mtgp_params_load(str(f))
    assert ei.value.status == status


def test_params_load_missing_file(lib):
    with pytest.raises(mtgp.MtgpError) as ei:
        mtgp.mtgp_params_load("/nonexistent/params.txt")
    assert ei.value.status == 6


def test_params_create_explicit_n_and_mask(lib):
    # the literal N = 727 row: Mexp 23209 with N = 727 and the mask of N = 726
    o = oracle.params_generate(23209, workloads.PARAM_SEED)
    p = mtgp.mtgp_params_create(23209, o.pos, o.sh1, o.sh2, list(o.rec_tbl), list(o.tmp_tbl),
                                n=727, mask=o.mask)
    d = mtgp.mtgp_params_get(p)
    assert d["n"] == 727 and d["mask"] == o.mask == 0xFF800000


def test_params_generate_rejects_bad_mexp(lib):
    for mexp in (32, 64, 10):
        with pytest.raises(mtgp.MtgpError):
            mtgp.mtgp_params_generate(mexp, 1)


def test_last_error_is_thread_local_message(lib):
    with pytest.raises(mtgp.MtgpError) as ei:
        mtgp.mtgp_params_generate(64, 1)
    assert "64" in str(ei.value)


# --------------------------------------------------------------------------
# Comparison generator (include/mtgp_mt.h): host-only parameter code
# --------------------------------------------------------------------------
def test_mt_params_mt19937_matches_oracle(lib):
    import oracle.mt as omt
    assert mtgp.mtgp_mt_params_mt19937().as_dict() == omt.params_mt19937().as_dict()


@pytest.mark.parametrize("p", [521, 3217, 4423, 19937, 44497])
@pytest.mark.parametrize("seed", [0, 7, 0xC0FFEE])
def test_mt_params_generate_matches_oracle(lib, p, seed):
    import oracle.mt as omt
    assert mtgp.mtgp_mt_params_generate(p, seed).as_dict() == omt.params_generate(p, seed).as_dict()


def test_mt_params_generate_rejects_small_exponent(lib):
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_mt_params_generate(32, 1)
