"""C ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and rejects bad patterns on the host before touching CUDA."""
import os
import re

import numpy as np
import pytest

from paper_2309_11488_gb300 import opm, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "opm_bsr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(opm_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2309_11488_gb300 import build
    build.build()


def test_every_declared_symbol_is_exported():
    syms = header_symbols()
    assert "opm_bsr_create" in syms and "opm_bicgstab_solve" in syms and "opm_ilu0_factor" in syms
    L = opm.lib()
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(opm.EXPORTS) == sorted(syms)


def test_status_strings():
    assert opm.opm_status_str(0) == "ok"
    assert "singular" in opm.opm_status_str(opm.OPM_ERR_ZERO_PIVOT)
    assert opm.opm_status_str(42) == "unknown status"


def test_options_default():
    o = opm.opm_options_default()
    assert o.schedule == 0 and o.precision == 0 and o.debug_skip_item == -1 and o.chunk == 0


def test_iterative_sweep_options_are_bounded_on_the_host():
    s = synth.config1()
    for kw in ({"cp_sweeps": -1}, {"tri_sweeps": -1}, {"cp_sweeps": 4097}, {"tri_sweeps": 65}):
        st, h = opm.opm_bsr_create(s.nb, s.rowptr, s.colidx, s.vals, opm.opm_options_default(**kw), check=False)
        assert st == opm.OPM_ERR_ARG and h is None


def _create(nb, rp, ci, vals, **kw):
    return opm.opm_bsr_create(nb, np.asarray(rp, np.int32), np.asarray(ci, np.int32),
                              np.asarray(vals, np.float64), opm.opm_options_default(**kw), check=False)


def test_pattern_errors_are_found_on_the_host():
    s = synth.config1()
    # unsorted columns in row 3
    ci = s.colidx.copy()
    a = s.rowptr[3]
    ci[a], ci[a + 1] = ci[a + 1], ci[a]
    st, h = _create(s.nb, s.rowptr, ci, s.vals)
    assert st == opm.OPM_ERR_PATTERN and h is None and opm.opm_last_error_row(None) == 3
    # column out of range in row 10
    ci = s.colidx.copy()
    ci[s.rowptr[11] - 1] = s.nb
    st, h = _create(s.nb, s.rowptr, ci, s.vals)
    assert st == opm.OPM_ERR_PATTERN and opm.opm_last_error_row(None) == 10
    # decreasing rowptr
    rp = s.rowptr.copy()
    rp[5] = rp[6] + 1
    st, h = _create(s.nb, rp, s.colidx, s.vals)
    assert st == opm.OPM_ERR_PATTERN
    # a row without its diagonal: row 0 of a 2-row system holds only column 1
    st, h = _create(2, [0, 1, 3], [1, 0, 1], np.ones(27))
    assert st == opm.OPM_ERR_NO_DIAG and opm.opm_last_error_row(None) == 0
    # duplicate column
    st, h = _create(2, [0, 2, 3], [0, 0, 1], np.ones(27))
    assert st == opm.OPM_ERR_PATTERN


def test_bad_arguments():
    s = synth.config1()
    st, h = _create(-1, [0], [], [])
    assert st == opm.OPM_ERR_ARG
    st, h = _create(s.nb, s.rowptr, s.colidx, s.vals, schedule=9)
    assert st == opm.OPM_ERR_ARG
    st, h = _create(s.nb, s.rowptr, s.colidx, s.vals, precision=5)
    assert st == opm.OPM_ERR_ARG
    # nb beyond the row limit is refused before any array is read
    # (non-null arrays, so that only the size can be the reason)
    st, h = _create(opm.OPM_MAX_ROWS + 1, [0, 1], [0], np.zeros(9))
    assert st == opm.OPM_ERR_ARG
    st, perm, info = opm.opm_bsr_analyse(opm.OPM_MAX_ROWS + 1, np.array([0, 1], np.int32), np.zeros(1, np.int32),
                                         "level")
    assert st == opm.OPM_ERR_ARG and perm.size == 0


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2309_11488_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "oracle.c" not in txt and "liboracle" not in txt, f


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the sizes and field offsets a C
    compiler gives the header's structures (plain gcc on this host)."""
    import ctypes
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    checks = {"opm_options": opm.opm_options, "opm_info": opm.opm_info, "opm_timing": opm.opm_timing,
              "opm_tune_entry": opm.opm_tune_entry, "opm_tune_report": opm.opm_tune_report,
              "opm_analysis_info": opm.opm_analysis_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "opm_bsr.h"', 'int main(void) {']
    for cname, cls in checks.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append('  return 0; }')
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {}
    for ln in out:
        if ln:
            parts = ln.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, cls in checks.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_autotune_rejects_bad_arguments_on_the_host():
    s = synth.config1()
    st, kw, cands, best = opm.autotune(-1, s.rowptr, s.colidx, s.vals, np.zeros(3))
    assert st == opm.OPM_ERR_ARG and cands == [] and best == -1
    st, kw, cands, best = opm.autotune(s.nb, s.rowptr, s.colidx, s.vals, np.zeros(3 * s.nb), maxit=-1)
    assert st == opm.OPM_ERR_ARG
    st, kw, cands, best = opm.autotune_batch([], maxit=10)
    assert st == opm.OPM_ERR_ARG


def test_jacobi_create_needs_a_partition():
    import ctypes
    s = synth.config1()
    out = ctypes.c_void_p()
    st = opm.lib().opm_bsr_create_jacobi(s.nb, s.rowptr.ctypes.data, s.colidx.ctypes.data, s.vals.ctypes.data,
                                         None, None, ctypes.byref(out))
    assert st == opm.OPM_ERR_ARG and not out.value


# ------------------------------------------------- host analysis vs the oracle

ANALYSE_CASES = {
    "c1": synth.config1,
    "c2": synth.config2,
    "ragged33": lambda: synth.random_pattern_system(33, 3, 41),
    "long_rows": lambda: synth.random_pattern_system(70, 20, 42),
    "dense40": lambda: synth.random_pattern_system(40, 0, 43, dense=True),
    "chain": lambda: synth.chain_system(100),
    "tree": lambda: synth.tree_system(300, 44),
}


@pytest.mark.parametrize("schedule", ["natural", "level", "colour", "colour_sl", "colour_kempe"])
@pytest.mark.parametrize("name", list(ANALYSE_CASES))
def test_library_analysis_matches_the_oracle_schedule(name, schedule):
    """The library's host analysis (no GPU) orders the rows exactly as the
    oracle's independent implementation of the same rules, with the same
    number of levels or colours."""
    import oracle as O
    s = ANALYSE_CASES[name]()
    st, perm, info = opm.opm_bsr_analyse(s.nb, s.rowptr, s.colidx, schedule)
    assert st == opm.OPM_OK
    ref, nsets = O.schedule_perm(s.nb, s.rowptr, s.colidx, schedule)
    np.testing.assert_array_equal(perm, ref)
    assert info.nsets == nsets and info.schedule == opm.SCHEDULES[schedule]
    assert info.nnzb_kept == s.nnzb and info.nnzb_lower + info.nnzb_upper == s.nnzb - s.nb
    if schedule != "natural":
        assert info.nphases == nsets


@pytest.mark.parametrize("schedule", ["level", "colour_kempe"])
def test_library_analysis_of_a_block_jacobi_pattern_matches_the_oracle(schedule):
    import oracle as O
    s = synth.config2()
    part = synth.partition_grid(s, 12)
    st, perm, info = opm.opm_bsr_analyse(s.nb, s.rowptr, s.colidx, schedule, part=part)
    assert st == opm.OPM_OK
    jrp, jci = O.jacobi_pattern(s.nb, s.rowptr, s.colidx, s.vals, part)[:2]
    ref, nsets = O.schedule_perm(s.nb, jrp, jci, schedule)
    np.testing.assert_array_equal(perm, ref)
    assert info.nsets == nsets and info.nnzb_kept == int(jrp[-1])


def test_library_analysis_reports_pattern_errors():
    s = synth.config1()
    ci = s.colidx.copy()
    a = s.rowptr[3]
    ci[a], ci[a + 1] = ci[a + 1], ci[a]
    st, perm, info = opm.opm_bsr_analyse(s.nb, s.rowptr, ci, "colour")
    assert st == opm.OPM_ERR_PATTERN and opm.opm_last_error_row(None) == 3
    st, _, _ = opm.opm_bsr_analyse(s.nb, s.rowptr, s.colidx, 99)
    assert st == opm.OPM_ERR_ARG
    st, perm, info = opm.opm_bsr_analyse(0, np.zeros(1, np.int32), np.zeros(0, np.int32), "colour")
    assert st == opm.OPM_OK and perm.size == 0 and info.nsets == 0


SWEEP = [(nb, extra, frac) for nb in (1, 2, 5, 31, 32, 33, 64, 97, 200) for extra, frac in ((0, 0.0), (1, 0.5),
                                                                                       (3, 0.0), (8, 0.7))]


@pytest.mark.parametrize("nb,extra,frac", SWEEP)
def test_library_analysis_matches_the_oracle_on_random_patterns(nb, extra, frac):
    """Seeded random patterns, symmetric and not, sized around the 32-row
    slices: every schedule's permutation and set count equal the oracle's."""
    import oracle as O
    s = synth.one_way_system(synth.random_pattern_system(nb, extra, 1000 + nb * 10 + extra), frac, nb + extra)
    rowptr, colidx = s.rowptr, s.colidx
    for schedule in ("natural", "level", "colour", "colour_sl", "colour_kempe"):
        st, perm, info = opm.opm_bsr_analyse(nb, rowptr, colidx, schedule)
        assert st == opm.OPM_OK, schedule
        ref, nsets = O.schedule_perm(nb, rowptr, colidx, schedule)
        np.testing.assert_array_equal(perm, ref, err_msg=schedule)
        assert info.nsets == nsets, schedule
        assert info.nnzb_kept == rowptr[-1] and info.nnzb_lower + info.nnzb_upper == rowptr[-1] - nb


def test_constants_match_the_header(tmp_path):
    """Status codes, schedules, precisions, sweep modes, kernel indices and
    the tuner's table size: the binding's values are the header's (plain gcc
    on this host)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    want = {f"OPM_{k}": getattr(opm, f"OPM_{k}") for k in
            ("OK", "NOT_CONVERGED", "ERR_ARG", "ERR_PATTERN", "ERR_NO_DIAG", "ERR_ZERO_PIVOT", "ERR_BREAKDOWN",
             "ERR_NONFINITE", "ERR_OOM", "ERR_TIMEOUT", "ERR_CUDA", "TUNE_MAX", "MAX_ROWS")}
    want.update({f"OPM_SCHED_{k.upper()}": v for k, v in opm.SCHEDULES.items()})
    want.update({"OPM_PREC_FP64": opm.PRECISIONS["fp64"], "OPM_PREC_FP32_FACTORS": opm.PRECISIONS["fp32"]})
    want.update({f"OPM_SWEEP_{k.upper()}": v for k, v in opm.SWEEPS.items()})
    want.update({f"OPM_KERNEL_{k.upper()}": q for q, k in enumerate(opm.KERNELS)})
    want["OPM_KERNEL_COUNT"] = len(opm.KERNELS)
    lines = ['#include <stdio.h>', '#include "opm_bsr.h"', 'int main(void) {']
    lines += [f'  printf("{name} %d\\n", (int)({name}));' for name in want]
    lines.append('  return 0; }')
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "consts"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(ln.split() for ln in subprocess.check_output([str(exe)], text=True).splitlines() if ln)
    for name, v in want.items():
        assert int(got[name]) == v, name


def test_missing_library_fails_loudly():
    """Without the compiled library the binding raises ImportError on first
    use (no CPU fallback): checked in a fresh process pointed at a path that
    does not exist."""
    import subprocess
    import sys
    code = ("import numpy as np\n"
            "from paper_2309_11488_gb300 import opm, synth\n"
            "opm.LIB_PATH = '/nonexistent/libopm_bsr.so'\n"
            "opm._lib = None\n"
            "s = synth.config1()\n"
            "for call in (lambda: opm.lib(), lambda: opm.Solver(s.nb, s.rowptr, s.colidx, s.vals)):\n"
            "    try:\n"
            "        call()\n"
            "    except ImportError as e:\n"
            "        assert 'no CPU fallback' in str(e)\n"
            "    else:\n"
            "        raise SystemExit('no error')\n"
            "print('ok')\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stderr[-2000:]


@pytest.mark.parametrize("schedule", ["level", "colour_kempe"])
def test_block_jacobi_analysis_takes_any_int32_labels(schedule):
    """Partition labels are arbitrary int32 values (negative, extreme,
    non-contiguous): only equality matters.  The analysis of a one-way
    pattern with such labels equals the oracle's, and relabelling the
    partitions changes nothing."""
    import oracle as O
    s = synth.one_way_system(synth.random_pattern_system(240, 4, 51), 0.4, 52)
    base = (np.arange(s.nb) // 17).astype(np.int64)
    table = np.array([-2**31, 2**31 - 1, -7, 0, 123456789, -1, 5, 2**30, -2**30, 77, 3, -3, 9, 11, 13],
                     dtype=np.int64)
    part = table[base % len(table)].astype(np.int32)
    st, perm, info = opm.opm_bsr_analyse(s.nb, s.rowptr, s.colidx, schedule, part=part)
    assert st == opm.OPM_OK
    jrp, jci = O.jacobi_pattern(s.nb, s.rowptr, s.colidx, s.vals, part)[:2]
    ref, nsets = O.schedule_perm(s.nb, jrp, jci, schedule)
    np.testing.assert_array_equal(perm, ref)
    assert info.nsets == nsets and info.nnzb_kept == int(jrp[-1])
    st2, perm2, info2 = opm.opm_bsr_analyse(s.nb, s.rowptr, s.colidx, schedule, part=(base % len(table)).astype(np.int32))
    assert st2 == opm.OPM_OK and np.array_equal(perm2, perm) and info2.nnzb_kept == info.nnzb_kept


def test_the_c_abi_from_plain_c(tmp_path):
    """A C program compiled against include/opm_bsr.h and linked with the
    library runs the host-only analysis of a 2x2 grid: levels 0, 1, 1, 2
    and colours 0, 1, 1, 0 give the permutations below (set-major, closed
    rows first inside a set), the binding agrees line by line, and a
    missing diagonal is reported with its row."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    libdir = os.path.dirname(opm.LIB_PATH)
    exe = tmp_path / "analyse_grid"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "analyse_grid.c"),
                           "-L", libdir, "-lopm_bsr", f"-Wl,-rpath,{libdir}", "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    lines = out.stdout.splitlines()
    # the binding gives the same analysis
    rp = np.array([0, 3, 6, 9, 12], np.int32)
    ci = np.array([0, 1, 2, 0, 1, 3, 0, 2, 3, 1, 2, 3], np.int32)
    for line, schedule in zip(lines[:2], ("level", "colour")):
        st, perm, info = opm.opm_bsr_analyse(4, rp, ci, schedule)
        assert line == (f"ok schedule={info.schedule} nsets={info.nsets} lower={info.nnzb_lower} "
                        f"upper={info.nnzb_upper} perm={','.join(str(v) for v in perm)}")
    assert lines[0].endswith("nsets=3 lower=4 upper=4 perm=0,1,2,3")
    # colour 0 = {0, 3}, both with a neighbour in colour 1 (open): natural order; then {1, 2}
    assert lines[1].startswith("ok schedule=3 nsets=2") and lines[1].endswith("perm=0,3,1,2")
    assert lines[2] == "missing diagonal block row=1"


def _one_error(s, kind, row):
    """s's pattern with exactly one error of `kind` planted in `row`."""
    rp, ci = s.rowptr.copy(), s.colidx.copy()
    a, b = int(rp[row]), int(rp[row + 1])
    if kind == "unsorted":
        ci[a], ci[a + 1] = ci[a + 1], ci[a]
    elif kind == "duplicate":
        ci[a + 1] = ci[a]
    elif kind == "out_of_range":
        ci[b - 1] = s.nb + 5
    elif kind == "negative":
        ci[a] = -1
    elif kind == "no_diagonal":
        d = a + int(np.nonzero(ci[a:b] == row)[0][0])
        # replace the diagonal by a column the row lacks, keeping the row sorted
        free = sorted(set(range(s.nb)) - set(ci[a:b].tolist()))
        ci[d] = min(free, key=lambda c: abs(c - row))
        ci[a:b] = np.sort(ci[a:b])
    return rp, ci


@pytest.mark.parametrize("kind,status", [("unsorted", "PATTERN"), ("duplicate", "PATTERN"),
                                         ("out_of_range", "PATTERN"), ("negative", "PATTERN"),
                                         ("no_diagonal", "NO_DIAG")])
def test_a_single_pattern_error_is_reported_with_its_row(kind, status):
    """One error planted in a random row of several seeded patterns: the
    host analysis returns its status and names that row, for every
    schedule."""
    rng = np.random.default_rng(7)
    want = getattr(opm, f"OPM_ERR_{status}")
    for seed in range(4):
        s = synth.random_pattern_system(90, 3, 300 + seed)
        rows = [i for i in range(s.nb) if s.rowptr[i + 1] - s.rowptr[i] >= 2]
        row = int(rng.choice(rows))
        rp, ci = _one_error(s, kind, row)
        for schedule in ("natural", "level", "colour_kempe"):
            st, perm, info = opm.opm_bsr_analyse(s.nb, rp, ci, schedule)
            assert st == want and opm.opm_last_error_row(None) == row, (kind, seed, row, schedule, st)


def test_binding_defaults_are_the_papers_stopping_rule():
    """The binding's default rtol and maxit are the stopping rule printed in
    the paper (tests/golden/paper_facts.txt: relative reduction 0.01, at
    most 200 iterations)."""
    import inspect
    facts = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_facts.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                facts[k] = float(v)
    for fn in (opm.Solver.solve, opm.Batch.solve, opm.opm_bicgstab_solve):
        sig = inspect.signature(fn).parameters
        assert sig["rtol"].default == facts["default_rtol"] and sig["maxit"].default == facts["default_maxit"], fn


def _update_products(nb, rowptr, colidx):
    """Brute-force count of ILU0's update products on a pattern (Algorithm
    2's inner loop): for every block (i, k) with k < i, the j > k present in
    both row i and row k."""
    rows = [set(colidx[rowptr[i]:rowptr[i + 1]].tolist()) for i in range(nb)]
    return sum(1 for i in range(nb) for k in rows[i] if k < i for j in rows[i] if j > k and j in rows[k])


@pytest.mark.parametrize("schedule", ["natural", "level", "colour_kempe"])
def test_kept_analysis_matches_the_one_shot_analysis(schedule):
    """opm_analysis_create (host only) keeps the analysis opm_bsr_analyse
    computes: the same permutation and counts; its update-product count
    equals a brute-force count on the permuted pattern."""
    import oracle as O
    s = synth.one_way_system(synth.random_pattern_system(150, 4, 77), 0.4, 78)
    st, perm, info = opm.opm_bsr_analyse(s.nb, s.rowptr, s.colidx, schedule)
    assert st == opm.OPM_OK
    with opm.Analysis(s.nb, s.rowptr, s.colidx, schedule) as an:
        np.testing.assert_array_equal(an.permutation(), perm)
        assert (an.nb, an.nnzb) == (s.nb, s.nnzb)
        for f in ("schedule", "nsets", "nphases", "nnzb_kept", "nnzb_lower", "nnzb_upper", "nupdates"):
            assert getattr(an.info, f) == getattr(info, f), f
    prow, pcol, _ = O.permute(s.nb, s.rowptr, s.colidx, s.vals, perm)
    assert info.nupdates == _update_products(s.nb, prow, pcol) > 0


def test_kept_analysis_reports_pattern_errors_and_bad_arguments():
    s = synth.config1()
    ci = s.colidx.copy()
    a = s.rowptr[5]
    ci[a] = ci[a + 1]  # duplicate column in row 5
    with pytest.raises(opm.OpmError) as e:
        opm.Analysis(s.nb, s.rowptr, ci, "colour")
    assert e.value.status == opm.OPM_ERR_PATTERN and opm.opm_last_error_row(None) == 5
    with pytest.raises(opm.OpmError):
        opm.Analysis(s.nb, s.rowptr, s.colidx, 99)
    import ctypes
    out = ctypes.c_void_p()
    assert opm.lib().opm_bsr_create_from_analysis(None, s.vals.ctypes.data, None, ctypes.byref(out)) == \
        opm.OPM_ERR_ARG and not out.value
