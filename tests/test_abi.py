"""The C ABI without a GPU: the library loads, exports every function include/qrng.h declares,
and its pure host functions agree with the oracle. No compute call is made here."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"QRNG_API\s+[\w\s\*]*?\b(qrng_\w+)\s*\(", txt)
    return names


def test_header_declares_entry_points():
    names = _declared()
    assert "qrng_minentropy" in names and "qrng_toeplitz_extract" in names
    assert len(names) == len(set(names))


def test_library_exports_every_declared_symbol(qlib):
    import ctypes

    import paper_2011_04130_gb300 as q

    lib = q.load_library()
    for name in _declared():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)
    assert set(_declared()) == set(q.EXPORTED)


def test_no_internal_symbols_exported(qlib):
    import subprocess

    import paper_2011_04130_gb300 as q

    out = subprocess.run(["nm", "-D", "--defined-only", q.LIB_PATH], capture_output=True, text=True).stdout
    syms = [l.split()[-1] for l in out.splitlines() if " T " in l]
    assert sorted(syms) == sorted(_declared())


@pytest.mark.parametrize("n,h,bits,eps", [(1024, 8.0, 8, 2.0 ** -10), (4096, 4.0, 8, 1.0), (1000, 3.3, 5, 0.5),
                                          (100, 0.1, 8, 1e-6), (65536, 4.4567, 8, 1.0), (1 << 20, 11.9, 16, 1e-9)])
def test_output_length_matches_oracle(qlib, oracle_mod, n, h, bits, eps):
    import paper_2011_04130_gb300 as q

    assert q.qrng_output_length(n, h, bits, eps) == oracle_mod.output_length(n, h, bits, eps)


@pytest.mark.parametrize("n,m,form", [(10, 4, 0), (10, 10, 0), (10, 4, 1), (10, 10, 1), (5, 0, 0), (1 << 27, 3, 0)])
def test_seed_bits(qlib, oracle_mod, n, m, form):
    import paper_2011_04130_gb300 as q

    valid = m >= 1 and ((form == 0 and m <= n) or (form == 1 and m < n)) and n <= (1 << 26)
    want = oracle_mod.seed_bits(n, m, form) if valid else 0
    assert q.qrng_seed_bits(n, m, form) == want


def test_create_rejects_bad_device(qlib):
    import paper_2011_04130_gb300 as q

    with pytest.raises(q.QrngError):
        q.Context(10_000)


def test_status_strings(qlib):
    import paper_2011_04130_gb300 as q

    assert q.qrng_status_string(q.QRNG_OK) == "QRNG_OK"
    assert q.qrng_status_string(q.QRNG_ENOTSUP) == "QRNG_ENOTSUP"


def test_product_package_does_not_import_oracle():
    """The product path never reaches the oracle: no reference to it in the package sources."""
    pkg = os.path.join(ROOT, "paper_2011_04130_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in txt and "qrng_oracle" not in txt and "liboracle" not in txt, fn


def test_fft32_terms_bound_is_percivals(qlib):
    """The proven term count of the FP32 route, recomputed here from the bound's statement: the
    largest T with T sqrt((2S-1) S) (eps_k + T u) <= 0.45, eps_k = (1+u)^{3k} (1+sqrt5 u)^{3k+1}
    (1+u/2)^{3k} - 1, k = log2(2S), u = 2^-24 (evaluated with exact rationals)."""
    from fractions import Fraction as F
    import math

    import paper_2011_04130_gb300 as q

    for S in (2048, 4096, 8192):
        k = S.bit_length()  # log2(2S)
        u = 2.0 ** -24
        eps = math.expm1(3 * k * math.log1p(u) + (3 * k + 1) * math.log1p(math.sqrt(5) * u) +
                         3 * k * math.log1p(u / 2))
        per = math.sqrt((2 * S - 1) * S)
        T = max(t for t in range(1, 100) if t * per * (eps + t * u) <= 0.45)
        assert q.qrng_fft32_terms_bound(S) == T, S
        assert T * per * (eps + T * u) < F(1, 2)
    assert [q.qrng_fft32_terms_bound(S) for S in (2048, 4096, 8192)] == [16, 8, 3]
    assert q.qrng_fft32_terms_bound(1024) == 0 and q.qrng_fft32_terms_bound(5000) == 0


_C_TYPES = {"double": 8, "uint64_t": 8, "int64_t": 8, "uint32_t": 4, "int32_t": 4, "int": 4}


def _header_structs():
    """Field lists (name, byte size, array length) of every typedef'd struct in include/qrng.h."""
    txt = open(os.path.join(ROOT, "include", "qrng.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", txt, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            m = re.match(r"((?:const\s+)?\w+\s*\**)\s*(.*)$", decl, flags=re.S)
            ctype, names = m.group(1), m.group(2)
            size = 8 if "*" in ctype else _C_TYPES[ctype.strip()]
            for item in names.split(","):
                am = re.match(r"(\w+)\s*(?:\[(\d+)\])?$", item.strip())
                fields.append((am.group(1), size, int(am.group(2) or 1)))
        out[name] = fields
    return out


def test_binding_structs_mirror_the_header():
    """Every struct the binding passes through the C ABI has the header's fields, in order, with
    the same sizes (a field added on one side only would shift every later field)."""
    import ctypes

    import paper_2011_04130_gb300 as q

    structs = _header_structs()
    pairs = {"qrng_hmin_report": q.HminReport, "qrng_request": q.Request, "qrng_stats": q.Stats,
             "qrng_karatsuba_plan_info": q.KaratsubaPlan}
    assert set(pairs) <= set(structs)
    for cname, py in pairs.items():
        got = []
        for fname, ftype in py._fields_:
            length = getattr(ftype, "_length_", 1)
            elem = getattr(ftype, "_type_", ftype) if length > 1 else ftype
            got.append((fname, ctypes.sizeof(elem), length))
        assert got == structs[cname], cname
