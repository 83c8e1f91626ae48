"""The C ABI library: builds for sm_103a, loads, exports every symbol that
include/smc.h declares, and its host-side collocation data agree with the
oracle's independent construction.  No GPU needed."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import sdc
from paper_1309_7327_gb300 import build as B
from paper_1309_7327_gb300 import smc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "smc.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return smc.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(smc_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ("smc_create", "smc_rhs", "smc_sdc_step", "smc_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (smc_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)
    assert sorted(smc.EXPORTS) == declared_functions()


def test_library_is_built_for_sm103a(lib):
    out = subprocess.run(["cuobjdump", "--list-elf", B.LIB], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_struct_layouts_match_c(tmp_path):
    """ctypes mirrors of the public structs have the C sizes and offsets."""
    src = tmp_path / "probe.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "smc.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(smc_grid),'
                   ' offsetof(smc_grid, dx), sizeof(smc_mechanism), offsetof(smc_mechanism, eta_ref),'
                   ' sizeof(smc_bc), sizeof(smc_stats), offsetof(smc_stats, ncells));return 0;}\n')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(smc.smc_grid), smc.smc_grid.dx.offset, ctypes.sizeof(smc.smc_mechanism),
            smc.smc_mechanism.eta_ref.offset, ctypes.sizeof(smc.smc_bc), ctypes.sizeof(smc.smc_stats),
            smc.smc_stats.ncells.offset]
    assert got == want


@pytest.mark.parametrize("nodes", [3, 5, 7])
def test_collocation_matches_oracle(lib, nodes):
    tau, S = smc.smc_collocation(nodes)
    assert np.abs(tau - sdc.gauss_lobatto(nodes)).max() < 1e-15
    assert np.abs(S - sdc.s_matrix(sdc.gauss_lobatto(nodes))).max() < 1e-14


@pytest.mark.parametrize("coarse,fine,repeat", [(3, 5, 1), (3, 9, 1), (5, 5, 1), (3, 2, 1),
                                                (5, 3, 1), (3, 3, 8), (3, 5, 2), (5, 3, 3)])
def test_multirate_collocation_matches_oracle(lib, coarse, fine, repeat):
    """Type (b) (repeat 1) and type (c) fine nodes and matrices."""
    t1, t2, S21, S22 = smc.smc_multirate_collocation(coarse, fine, repeat)
    a, b, S21o, S22o = sdc.mr_matrices(coarse, fine, repeat)
    assert np.abs(t1 - a).max() < 1e-15
    assert np.abs(t2 - b).max() < 1e-15
    assert np.abs(S21 - S21o).max() < 1e-14
    assert np.abs(S22 - S22o).max() < 1e-14


def test_collocation_rejects_bad_arguments(lib):
    with pytest.raises(smc.SmcError):
        smc.smc_collocation(1)
    with pytest.raises(smc.SmcError):
        smc.smc_multirate_collocation(3, 12)
    with pytest.raises(smc.SmcError):
        smc.smc_multirate_collocation(3, 3, 0)


def test_create_rejects_bad_mechanism_without_touching_the_gpu(lib):
    """Mass-unbalanced reactions are refused during host validation, before
    any device allocation."""
    from paper_1309_7327_gb300 import synth
    m = synth.make_mechanism(3, 2, 1)
    m.nu_r = m.nu_r.copy()
    m.nu_r[0, 0] += 1
    g = synth.single_box(8, 0.1)
    with pytest.raises(smc.SmcError) as e:
        smc.Smc(g, m)
    assert e.value.status == smc.SMC_ERR_ARG and "mass" in str(e.value)


def test_create_rejects_unsupported_boundaries_without_touching_the_gpu(lib):
    """Non-periodic y or z faces, or mixed x faces, are refused during host
    validation; outflow x needs at least 8 cells along x."""
    from paper_1309_7327_gb300 import synth
    m = synth.make_mechanism(3, 2, 1)
    g = synth.single_box(8, 0.1)
    P, O = smc.SMC_BC_PERIODIC, smc.SMC_BC_OUTFLOW
    for bc in (((P, O, P), (P, O, P)), ((O, P, P), (P, P, P)), ((P, P, 7), (P, P, 7))):
        with pytest.raises(smc.SmcError) as e:
            smc.Smc(g, m, bc=bc)
        assert e.value.status == smc.SMC_ERR_ARG and "boundar" in str(e.value)
    with pytest.raises(smc.SmcError) as e:
        smc.Smc(synth.single_box((6, 8, 8), 0.1), m, x_outflow=True)
    assert "8 cells" in str(e.value)


def test_create_rejects_bad_box_arrays_without_touching_the_gpu(lib):
    """An empty box list, a box outside the domain, overlapping boxes and a
    domain the boxes do not cover are refused during host validation."""
    import numpy as np
    from paper_1309_7327_gb300 import synth
    m = synth.make_mechanism(3, 2, 1)
    dx = (0.1, 0.1, 0.1)
    cases = {
        "no boxes": synth.Grid((8, 8, 8), dx, np.zeros((0, 3), np.int64), np.zeros((0, 3), np.int64)),
        "outside": synth.Grid((8, 8, 8), dx, np.array([[0, 0, 0]]), np.array([[8, 7, 7]])),
        "overlap": synth.Grid((8, 8, 8), dx, np.array([[0, 0, 0], [3, 0, 0]]),
                              np.array([[4, 7, 7], [7, 7, 7]])),
        "maps onto no box": synth.Grid((8, 8, 8), dx, np.array([[0, 0, 0]]),
                                       np.array([[3, 7, 7]])),
    }
    for what, g in cases.items():
        with pytest.raises(smc.SmcError) as e:
            smc.Smc(g, m)
        assert e.value.status == smc.SMC_ERR_ARG, what
        assert what in str(e.value) or what == "outside" and "outside" in str(e.value), \
            (what, str(e.value))


def test_create_rejects_more_species_than_the_limit_without_touching_the_gpu(lib):
    """64 species is the largest mechanism the kernels are built for; 65 is
    refused during host validation."""
    from paper_1309_7327_gb300 import synth
    m = synth.make_mechanism(65, 10, 3)
    with pytest.raises(smc.SmcError) as e:
        smc.Smc(synth.single_box(8, 0.1), m)
    assert e.value.status == smc.SMC_ERR_ARG
