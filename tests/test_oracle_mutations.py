"""Plant plausible mistakes in copies of the oracle's C source and check that the pins catch
every one of them (a pin set that a wrong oracle also passes would pin nothing)."""
import pytest

from pins import ALL_PINS

MUTATIONS = [
    ("precession sense reversed", [("(M[0] * c + M[1] * s)", "(M[0] * c - M[1] * s)"),
                                   ("(-M[0] * s + M[1] * c)", "(M[0] * s + M[1] * c)")]),
    ("RF matrix transposed", [("R[0][2] = -sp * sa;", "R[0][2] = sp * sa;"),
                              ("R[2][0] = sp * sa;", "R[2][0] = -sp * sa;"),
                              ("R[1][2] = cp * sa;", "R[1][2] = -cp * sa;"),
                              ("R[2][1] = -cp * sa;", "R[2][1] = cp * sa;")]),
    ("RF phase axis swapped", [("const double cp = cos(phi), sp = sin(phi);", "const double cp = sin(phi), sp = cos(phi);")]),
    ("RF 1-cos sign", [("R[0][1] = sp * cp * (1.0 - ca);", "R[0][1] = sp * cp * (1.0 + ca);")]),
    ("T1 recovery term dropped", [("M[2] * e1 + rho * (1.0 - e1)", "M[2] * e1")]),
    ("T2 decay uses T1", [("exp(-e->dt / t2)", "exp(-e->dt / t1)")]),
    ("off-resonance dropped", [("e->gz * z) + dw)", "e->gz * z))")]),
    ("wrong gradient axis", [("e->gy * y", "e->gy * x")]),
    ("demodulation sign", [("M[0] * cph + M[1] * sph", "M[0] * cph - M[1] * sph"),
                           ("M[1] * cph - M[0] * sph", "M[1] * cph + M[0] * sph")]),
    ("RF after precession", None),
    ("sample before the step", None),
]


def _reorder_rf_after(src):
    a = src.index("    if (e->rf_flip != 0.0) {")
    b = src.index("    /* Eq. 3.14 with the off-resonance")
    c = src.index("    return e->adc != 0;")
    return src[:a] + src[b:c] + src[a:b] + src[c:]


def _sample_first(src):
    # take the sample with the state before the event: apply the event after reading M
    old = "                if (apply_event(&ev[e], gamma, x[s], y[s], z[s], rho[s], t1[s], t2[s], dw[s], M)) {"
    new = ("                double Mprev[3] = {M[0], M[1], M[2]};\n"
           "                int sampled = apply_event(&ev[e], gamma, x[s], y[s], z[s], rho[s], t1[s], t2[s], dw[s], M);\n"
           "                double Msave[3] = {M[0], M[1], M[2]};\n"
           "                M[0] = Mprev[0]; M[1] = Mprev[1]; M[2] = Mprev[2];\n"
           "                if (sampled) {")
    src = src.replace(old, new)
    old2 = "                    ++j;\n                }\n"
    new2 = "                    ++j;\n                }\n                M[0] = Msave[0]; M[1] = Msave[1]; M[2] = Msave[2];\n"
    assert old2 in src
    return src.replace(old2, new2, 1)


@pytest.mark.parametrize("name,edits", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(name, edits, oracle_mod, tmp_path):
    src = oracle_mod.source()
    if name == "RF after precession":
        bad = _reorder_rf_after(src)
    elif name == "sample before the step":
        bad = _sample_first(src)
    else:
        bad = src
        for old, new in edits:
            assert old in bad, f"mutation anchor not found: {old}"
            bad = bad.replace(old, new)
    assert bad != src
    variant = oracle_mod.Variant(bad, str(tmp_path))
    caught = []
    for pin in ALL_PINS:
        try:
            pin(variant.simulate)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin caught the planted mistake: {name}"
