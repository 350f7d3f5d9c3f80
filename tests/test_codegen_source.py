"""The generator of per-segment kernels (N2) on host-built records, without a
GPU: the source holds one assignment per row from its folded constant, one
FMA per term with the coefficient as a hexadecimal literal and the unknown
from a register (solved in the same generated function of 32 rows) or from
shared memory (solved earlier), the undivided row's IEEE division, the row
ids it writes, and it compiles for sm_103a; bad records are refused."""
import re
import shutil
import subprocess

import numpy as np
import pytest


def records(nrows=80, K=4):
    rng = np.random.default_rng(5)
    row = 1000 + np.arange(nrows, dtype=np.int32)          # where x is written
    nn = np.zeros(nrows, np.int32)
    term = np.zeros((K, nrows, 4), np.int32)
    coef = {}
    for p in range(1, nrows):
        deps = [p - 1] + ([p - 40] if p >= 40 else [])
        for k, q in enumerate(deps):
            v = float(rng.uniform(-1, 1))
            bits = np.array([v], np.float64).view(np.int32)
            term[k, p] = (q, 0, bits[0], bits[1])
            coef[(p, q)] = v
        nn[p] = len(deps)
    nn[5] |= 1 << 30                                         # kept undivided
    diag = np.zeros((nrows, 2))
    diag[:, 0] = 4.0
    return row, nn, term, diag, coef


def test_source_structure():
    from paper_2103_11445_gb300 import binding as B
    row, nn, term, diag, coef = records()
    src = B.sptrsv_codegen_source_from_records(80, row, nn, term, diag)
    assert src.count("a = s0[") == 80
    fns = re.findall(r"__device__ __noinline__ void g(\d+)\(", src)
    assert fns == [str(f) for f in range(3)]                 # 32 + 32 + 16 rows
    # walk the rows in order and check every FMA against the records
    body = src.split("extern \"C\"")[0]
    rows = body.split("  a = s0[")[1:]
    for p, chunk in enumerate(rows):
        assert chunk.startswith(f"{p}];")
        fmas = re.findall(r"a = fma\(([^,]+), (v|xs)\[(\d+)\], a\);", chunk)
        p0 = 32 * (p // 32)
        deps = sorted(q for (pp, q) in coef if pp == p)       # oldest first
        assert len(fmas) == len(deps)
        for (lit, where, idx), q in zip(fmas, deps):
            assert float.fromhex(lit) == -coef[(p, q)]
            if q >= p0:
                assert where == "v" and int(idx) == q - p0
            else:
                assert where == "xs" and int(idx) == q
        assert f"x[{1000 + p}] = a;" in chunk
        assert ("__ddiv_rn(a, 0x1p+2)" in chunk) == (p == 5)


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="no CUDA compiler")
def test_source_compiles_for_sm_103a(tmp_path):
    from paper_2103_11445_gb300 import binding as B
    row, nn, term, diag, _ = records()
    src = B.sptrsv_codegen_source_from_records(80, row, nn, term, diag)
    f = tmp_path / "gen.cu"
    f.write_text(src)
    r = subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-c", str(f),
                        "-o", str(tmp_path / "gen.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]


def test_bad_records_are_refused():
    from paper_2103_11445_gb300 import binding as B
    row, nn, term, diag, _ = records()
    bad = term.copy()
    bad[0, 10, 0] = 10                                       # a row reading itself
    with pytest.raises(B.SptrsvError):
        B.sptrsv_codegen_source_from_records(80, row, nn, bad, diag)
    thick = nn.copy()
    with pytest.raises(B.SptrsvError):                       # 80 rows in 2 levels: not thin
        B.sptrsv_codegen_source_from_records(2, row, thick, term, diag)
