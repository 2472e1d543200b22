"""Host-side checks of the C-ABI library (no GPU): it loads, exports every
symbol include/gqt.h declares, and its host-only routines (lattice generator,
Bessel coefficients, expansion-length rule) agree with independent references."""
import os
import re

import numpy as np
import pytest
import scipy.special as sp

import gqt_synth as S

g = pytest.importorskip("paper_1705_01387_gb300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gqt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gqt_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = g.lib()
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if getattr(L, n, None) is None]
    assert not missing, missing


@pytest.mark.parametrize("kind,args,synth", [
    (g.GQT_LATTICE_HONEYCOMB, dict(L1=7, L2=5, t=-2.7, W=2.0, vacancy_frac=0.05, seed=99),
     lambda: S.honeycomb(7, 5, -2.7, 2.0, seed=99, vacancy_frac=0.05)),
    (g.GQT_LATTICE_SQUARE, dict(L1=6, L2=4, t=-1.0, W=4.0, seed=3), lambda: S.square(6, 4, -1.0, 4.0, seed=3)),
    (g.GQT_LATTICE_CHAIN, dict(L1=11, t=-1.0, W=4.0, seed=5), lambda: S.chain(11, -1.0, 4.0, seed=5)),
    (g.GQT_LATTICE_CUBIC, dict(L1=4, t=-1.0, W=16.5, seed=7), lambda: S.cubic(4, -1.0, 16.5, seed=7)),
])
def test_native_lattice_matches_generator(kind, args, synth):
    """The library's built-in lattices are the generator's, bit for bit."""
    out = g.gqt_generate_lattice(kind, **args)
    lat = synth()
    assert out["n"] == lat.n and out["K"] == lat.max_nb
    assert np.array_equal(out["nb_count"], lat.nb_count)
    assert np.array_equal(out["nb_idx"], lat.nb_idx)
    assert np.array_equal(out["hop_re"], lat.hop.real) and np.array_equal(out["hop_im"], lat.hop.imag)
    assert np.array_equal(out["onsite"], lat.onsite)
    assert np.array_equal(out["bond_dx"], lat.dx)
    assert out["volume"] == pytest.approx(lat.volume, rel=1e-15)
    assert out["length_x"] == pytest.approx(lat.length_x, rel=1e-15)


def test_vacancy_count_is_exact():
    out = g.gqt_generate_lattice(g.GQT_LATTICE_HONEYCOMB, L1=20, L2=20, t=-2.7, W=0.5, vacancy_frac=0.01, seed=1)
    dead = np.all(out["hop_re"] == 0.0, axis=1)
    assert dead.sum() >= round(0.01 * out["n"])


def test_library_bessel_matches_scipy():
    for x in (0.0, 1e-3, 0.37, 3.344, 7.08, 40.0, 410.0):
        J = g.gqt_bessel(x, 120)
        ref = sp.jv(np.arange(120), x)
        # the backward recurrence runs over ~x + 100 orders; allow its rounding to grow with x
        assert np.max(np.abs(J - ref)) < (5e-15 if x < 50 else 2e-14), x


def test_library_np_rule_matches_scipy():
    m = np.arange(800)
    for x in (0.5, 9.03 / 2.7, 9.555 * 2 / 2.7, 8.7675 * 2 / 2.7, 41.0):
        ref = 1 + int(np.max(m[np.abs(sp.jv(m, x)) >= 1e-15]))
        assert g.gqt_np_rule(x, 4096) == ref


def test_bad_arguments_return_status_not_abort():
    # built-in kind too small -> EINVAL through the host path (no device work)
    with pytest.raises(g.GqtError) as e:
        g.gqt_generate_lattice(g.GQT_LATTICE_CHAIN, L1=2)
    assert e.value.status == g.GQT_EINVAL
    with pytest.raises(g.GqtError):
        g.gqt_bessel(-1.0, 4)
