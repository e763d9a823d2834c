"""Source layout rules that keep the parity claims meaningful (no GPU): the oracle and the CUDA
path share no code, the product never reaches into the oracle, and the seeded input generators
hold no method arithmetic that either side could borrow."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2306_03651_gb300")


def files(top, exts):
    for d, _, names in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in names:
            if f.endswith(exts):
                yield os.path.join(d, f)


def code(path):
    """Source text without comments, docstrings or string literals (a crude strip, enough for
    include and import lines)."""
    text = open(path, encoding="utf-8").read()
    if path.endswith(".py"):
        text = re.sub(r'"""[\s\S]*?"""', "", text)
        text = re.sub(r"#.*", "", text)
    else:
        text = re.sub(r"/\*[\s\S]*?\*/", "", text)
        text = re.sub(r"//.*", "", text)
    return text


def test_product_does_not_use_the_oracle():
    for f in files(PKG, (".py", ".cu", ".cuh", ".c", ".h")):
        src = code(f)
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
        assert "oracle/" not in src and "liboracle" not in src, f


def test_oracle_includes_nothing_of_the_product():
    for f in files(os.path.join(ROOT, "oracle"), (".c", ".h", ".py")):
        src = code(f)
        for inc in re.findall(r'#include\s+"([^"]+)"', src):
            assert os.path.basename(inc) in ("oracle.h",), (f, inc)
        assert not re.search(r"^\s*(import|from)\s+paper_2306_03651_gb300\b", src, re.M), f
        assert "csrc" not in src and "libcen" not in src, f


def test_cuda_sources_include_only_their_own_headers_and_the_abi():
    own = {os.path.basename(f) for f in files(os.path.join(PKG, "csrc"), (".cuh", ".h"))} | {"cen.h"}
    for f in files(os.path.join(PKG, "csrc"), (".cu", ".cuh")):
        for inc in re.findall(r'#include\s+"([^"]+)"', code(f)):
            assert os.path.basename(inc) in own, (f, inc)


def test_input_generators_hold_no_method_arithmetic():
    """The generators draw graphs and raw random words; Philox, path counts, covers and bounds
    live only on the two sides that are compared."""
    gen = code(os.path.join(PKG, "inputs", "gen.c")) + code(os.path.join(PKG, "inputs", "__init__.py"))
    for word in ("philox", "sigma", "greedy", "rademacher", "amcera", "bound"):
        assert word not in gen.lower(), word
