import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter):
    """A few lines of parity counts (images and hit sets against the FP64 definition,
    finite differences), aggregated over the checks that ran."""
    try:
        from parity_rules import REPORT
    except Exception:
        return
    if not REPORT:
        return
    w = terminalreporter.write_line
    img = [st for kind, _, st in REPORT if kind == "image"]
    if img:
        worst = min(img, key=lambda st: st["frac_2e-4"])
        w(f"parity vs FP64 definition: {len(img)} image checks, {sum(st['rays'] for st in img)} rays; "
          f"channels within 2e-4 >= {worst['frac_2e-4']:.5f}; max error {max(st['max'] for st in img):.3g}; "
          f"pixels over 2e-4 {sum(st['px_over_2e-4'] for st in img)} (not near a face: "
          f"{sum(st['px_over_2e-4_not_near_face'] for st in img)}), over 1e-2 "
          f"{sum(st['px_over_1e-2'] for st in img)}, near-face pixels {sum(st['px_near_face'] for st in img)}")
    hits = [st for kind, _, st in REPORT if kind == "hits"]
    if hits:
        w(f"hit sets vs FP64 definition: {len(hits)} checks, {sum(st['pairs_f64'] for st in hits)} FP64 pairs, "
          f"grazing differences {sum(st['grazing_differences'] for st in hits)}, largest depth miss of a "
          f"GPU-only pair {max(st['max_depth_miss_gpu_only'] for st in hits):.2g}")
    for kind, label, st in REPORT:
        if kind == "fd" and not label.startswith("planted"):
            w(f"finite differences ({label}): {st['params']} parameters, error max {st['err_max']:.3g}, plain C9 "
              f"max {st['plain_c9_max']:.3g} ({st['plain_c9_ok']} within 1e-3); rays straddling a kink "
              f"{st['kinked']}, within FP32 rounding of one {st['near_kink']}, of {st['rays']}")
    for kind, label, st in REPORT:
        if kind == "grad":
            w(f"adjoint vs oracle ({label}): per element max / p99 / per tensor: " +
              ", ".join(f"{k} {v[0]:.2g}/{v[1]:.2g}/{v[2]:.2g}" for k, v in st.items()))
    prec = [(label, st) for kind, label, st in REPORT if kind == "precision"]
    if prec:
        w("payload precision vs FP64 oracle on the FP32 payload (max / p99.9 over channels): " +
          "; ".join(f"{label} {st['max']:.2g} / {st['p999']:.2g}" for label, st in prec))
