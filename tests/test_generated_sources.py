"""The per-class kernel translation units and the class registry are generated by
csrc/gen_kernels.py; the committed files must be exactly what it writes."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1305_3699_gb300", "csrc")


def _generator():
    spec = importlib.util.spec_from_file_location("gen_kernels", os.path.join(CSRC, "gen_kernels.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_generated_units_match_generator():
    g = _generator()
    expected = {}
    for L, (k, W, WX, variants) in g.CLASSES.items():
        expected[f"kern_{L}.cu"] = g.unit(L, k, W, WX, variants)
    for L, (k, W, WX, npt, nw) in g.BIG.items():
        expected[f"kern_{L}.cu"] = g.big_unit(L, k, W, WX, npt, nw)
    for name, text in expected.items():
        with open(os.path.join(CSRC, name)) as f:
            assert f.read() == text, name


def test_generated_classes_match_the_base_rule():
    from oracle import rns
    g = _generator()
    for L, (k, W, WX, _) in g.CLASSES.items():
        assert k == rns.class_k(L) and W == L // 32, L
    for L, (k, W, WX, _, _) in g.BIG.items():
        assert k == rns.class_k(L) and W == L // 32, L
