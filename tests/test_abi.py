"""The C ABI without a GPU: the library builds and loads, exports exactly the
entry points include/abcsmc.h declares, its structs have the layout a C
compiler gives them, argument checks answer before any device work, and the
binding has no fallback.  Also checks that the oracle and the CUDA path share
no code."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "abcsmc.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return G.lib()


def _declared():
    src = open(HEADER).read()
    return set(re.findall(r"^ABC_API[^(]*?\b(abc_\w+)\(", src, re.M))


def test_header_declarations_are_exported(lib):
    names = _declared()
    assert len(names) >= 26
    out = subprocess.run(["nm", "-D", "--defined-only", G.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert names <= exported, names - exported
    # nothing but the ABI leaks out of the library
    assert {e for e in exported if not e.startswith("abc_")} == set()
    assert set(G.EXPORTS) == names
    for n in names:
        getattr(lib, n)


def test_struct_layout_matches_c(lib):
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "abcsmc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(abc_config), offsetof(abc_config, population),
         offsetof(abc_config, seed), offsetof(abc_config, survival_alpha),
         offsetof(abc_config, max_redraw), sizeof(abc_gen_stats));
  printf("%zu %zu %zu %zu %zu %zu\n", offsetof(abc_gen_stats, eps), offsetof(abc_gen_stats, batches),
         offsetof(abc_gen_stats, ms_weights), offsetof(abc_gen_stats, beta_bf),
         offsetof(abc_config, beta_p2), offsetof(abc_config, max_total_batches));
  printf("%zu %zu %zu %zu\n", offsetof(abc_config, spec_batches), offsetof(abc_config, mcmc_s0),
         offsetof(abc_config, mcmc_adapt), offsetof(abc_gen_stats, mcmc_s));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        a, b, c = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines()
    got = [int(x) for x in a.split()] + [int(x) for x in b.split()] + [int(x) for x in c.split()]
    want = [ctypes.sizeof(G.AbcConfig), G.AbcConfig.population.offset, G.AbcConfig.seed.offset,
            G.AbcConfig.survival_alpha.offset, G.AbcConfig.max_redraw.offset,
            ctypes.sizeof(G.AbcGenStats), G.AbcGenStats.eps.offset, G.AbcGenStats.batches.offset,
            G.AbcGenStats.ms_weights.offset, G.AbcGenStats.beta_bf.offset,
            G.AbcConfig.beta_p2.offset, G.AbcConfig.max_total_batches.offset,
            G.AbcConfig.spec_batches.offset, G.AbcConfig.mcmc_s0.offset,
            G.AbcConfig.mcmc_adapt.offset, G.AbcGenStats.mcmc_s.offset]
    assert got == want


def test_defaults_and_argument_checks_without_gpu(lib):
    c = G.config()
    assert list(c.theta_hi) == [1, 100, 2, 1, 1, 1, 1, 2]  # Eq. 2
    assert c.survival_alpha == 0.5 and c.beta_mode == G.ABC_BETA_PAPER
    assert G.strerror(-1).startswith("invalid")
    h = ctypes.c_void_p()
    assert lib.abc_init(None, None, None, ctypes.byref(h)) == -1
    bad = G.config(n_particles=0)
    assert lib.abc_init(ctypes.byref(bad), None, None, ctypes.byref(h)) == -1
    bad = G.config(population=0)
    assert lib.abc_prior(ctypes.byref(bad), 10, None, None) == -1
    bad = G.config(beta_mode=G.ABC_BETA_FIXED, beta_b=0)
    assert lib.abc_init(ctypes.byref(bad), None, None, ctypes.byref(h)) == -1
    # real-shape rules: parameters outside their ranges
    for mode, p1, p2 in [(G.ABC_BETA_REAL, 0.0, 1.0), (G.ABC_BETA_REAL, 1.0, 2.0 ** 21),
                         (G.ABC_BETA_MEAN_VAR, 1.0, 0.01), (G.ABC_BETA_MEAN_VAR, 0.3, 0.0),
                         (G.ABC_BETA_MODE_CONC, 1.5, 3.0), (G.ABC_BETA_MODE_CONC, 0.5, 1.9),
                         (6, 0.5, 3.0)]:
        bad = G.config(beta_mode=mode, beta_p1=p1, beta_p2=p2)
        assert lib.abc_init(ctypes.byref(bad), None, None, ctypes.byref(h)) == -1, (mode, p1, p2)
    # the MCMC baseline: a positive finite step, a window >= 0, no surrogate
    assert G.config().mcmc_s0 > 0 and G.config().mcmc_adapt == 0
    for kw in (dict(mcmc_s0=0.0), dict(mcmc_s0=float("inf")), dict(mcmc_adapt=-1),
               dict(surrogate=1)):
        bad = G.config(beta_mode=G.ABC_STEP_MCMC, **kw)
        assert lib.abc_init(ctypes.byref(bad), None, None, ctypes.byref(h)) == -1, kw
    assert lib.abc_select_kth(None, 10, 1, None, None, 0, None) == -1
    assert lib.abc_select_scratch_bytes(1 << 20) > 0
    assert lib.abc_weights_scratch_bytes(4096, 4096) >= 4096 * 9 * 4


def test_binding_has_no_fallback(monkeypatch):
    monkeypatch.setattr(G, "_lib", None)
    monkeypatch.setattr(G, "LIB_PATH", "/nonexistent/libabcsmc.so")
    with pytest.raises(ImportError):
        G.lib()


def test_oracle_and_cuda_path_share_no_code():
    pkg = os.path.join(ROOT, "paper_2106_15508_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, re.M), f
                assert "abc_oracle" not in txt and "liboracle" not in txt, f
    osrc = open(os.path.join(ROOT, "oracle", "abc_oracle.c")).read()
    assert "#include \"" not in osrc  # only system headers
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2106_15508_gb300" not in txt, f
