"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer (CPU only).

Two builds are made in a temporary directory and exercised in a child
process that preloads the ASan runtime:

* the plain C oracle, driven through every entry point (weight matrix,
  exhaustive, branch-and-bound and EffBW decisions, score of a tuple,
  automorphism count) on random small instances, including malformed
  graphs, patterns and budgets;
* the library's host translation units (C ABI, serving, simulator, EffBW
  tables) compiled with both sanitizers and linked with the unmodified CUDA
  objects, driven through the calls that need no GPU: pattern analysis of
  random and malformed application graphs, Eq. 2 predictions inside and
  outside the supported link counts, the version string and the
  context-creation error text.

Any sanitizer report ends the child with a non-zero status.  Device code is
not instrumented here (compute-sanitizer is not used).
"""

import os
import shutil
import subprocess
import sys
import textwrap

import pytest

from oracle import oracle as O
from paper_2110_03214_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-g", "-O1"]


def _asan_runtime():
    if shutil.which("gcc") is None:
        return None
    path = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


pytestmark = pytest.mark.skipif(_asan_runtime() is None, reason="gcc with the ASan runtime is needed")


def _run_child(script, tmp_path):
    env = dict(os.environ)
    env["LD_PRELOAD"] = _asan_runtime()
    env["ASAN_OPTIONS"] = "detect_leaks=0:abort_on_error=0:exitcode=23"
    env["UBSAN_OPTIONS"] = "print_stacktrace=1:halt_on_error=1:exitcode=24"
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    path = tmp_path / "child.py"
    path.write_text(textwrap.dedent(script))
    proc = subprocess.run([sys.executable, str(path)], env=env, capture_output=True, text=True, timeout=600)
    report = proc.stdout[-4000:] + proc.stderr[-4000:]
    assert proc.returncode == 0, report
    assert "runtime error" not in proc.stderr and "AddressSanitizer" not in proc.stderr, report
    assert "child ok" in proc.stdout, report


def test_oracle_under_sanitizers(tmp_path):
    so = tmp_path / "liboracle_san.so"
    O.build(force=True, extra_flags=tuple(SAN), out=str(so))
    _run_child(
        f"""
        import numpy as np
        from oracle import oracle as O
        from paper_2110_03214_gb300 import workloads as W

        lib = O.load({str(so)!r})
        rng = W.Rng(31337, 5)
        calls = 0
        for trial in range(120):
            n = int(rng.integers(1, 12, 1)[0])
            pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
            keep = rng.uniform(len(pairs)) < 0.45
            u = np.asarray([p[0] for p, k in zip(pairs, keep) if k], np.int32)
            v = np.asarray([p[1] for p, k in zip(pairs, keep) if k], np.int32)
            w = rng.integers(1, 60, u.shape[0]).astype(np.int32)
            fill = 12 if trial % 5 == 0 else 0
            inst = O.Instance(n, u, v, w, fill, lib=lib)
            busy = rng.uniform(n) < 0.2
            k = int(rng.integers(1, min(n, 6), 1)[0])
            p = W.random_pattern(rng, k, 0.4, connected=bool(trial % 3))
            al, be = (int(x) for x in rng.integers(-2, 2, 2))
            budget = int(rng.integers(0, 1, 1)[0]) * 50
            d = inst.decide(busy, k, p.a, p.b, al, be, max_maps=budget)
            b = inst.decide_bounded(busy, k, p.a, p.b, al, be)
            e = inst.decide_effbw(busy, k, p.a, p.b)
            O.aut_count(k, p.a, p.b, lib=lib)
            calls += 4
            if d.status == O.STATUS_OK:
                assert (b.score, b.tuple) == (d.score, d.tuple)
        # malformed inputs take the error paths
        for bad in ((3, [0], [0], [5]), (3, [0], [3], [5]), (3, [0, 0], [1, 1], [5, 5]), (2, [0], [1], [0])):
            n, u, v, w = bad
            try:
                O.Instance(n, np.asarray(u, np.int32), np.asarray(v, np.int32), np.asarray(w, np.int32), lib=lib)
            except ValueError:
                calls += 1
        inst = O.Instance(4, np.asarray([0, 1], np.int32), np.asarray([1, 2], np.int32), np.asarray([5, 7], np.int32), lib=lib)
        for k, a, b in ((2, [0], [0]), (2, [0], [2]), (2, [0, 0], [1, 1]), (5, [0], [1]), (40, [], [])):
            d = inst.decide(np.zeros(4, bool), k, np.asarray(a, np.int32), np.asarray(b, np.int32))
            assert d.status != O.STATUS_OK
            calls += 1
        print("child ok", calls)
        """,
        tmp_path,
    )


def test_library_host_code_under_sanitizers(tmp_path):
    B.build()
    cuda = B._cuda_home()
    objs = []
    for src in sorted(os.listdir(B.CSRC)):
        stem, ext = os.path.splitext(src)
        if ext == ".cpp":
            obj = tmp_path / (stem + ".o")
            subprocess.check_call(["g++", "-std=c++17", "-fPIC", *SAN, "-c", os.path.join(B.CSRC, src), "-o", str(obj),
                                   "-I", B.CSRC, "-I", B.INCLUDE, "-I", os.path.join(cuda, "include")])
            objs.append(str(obj))
        elif ext == ".cu":
            objs.append(os.path.join(B.BUILD, stem + ".o"))
    so = tmp_path / "libmapa_san.so"
    lib64 = os.path.join(cuda, "lib64")
    subprocess.check_call(["g++", "-shared", *SAN, "-o", str(so), *objs, "-L", lib64, "-lcudart",
                           f"-Wl,-rpath,{lib64}"])
    _run_child(
        f"""
        import ctypes
        import itertools
        import numpy as np
        from paper_2110_03214_gb300 import workloads as W

        lib = ctypes.CDLL({str(so)!r})
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.mapa_pattern_analyze.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p,
                                             ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32),
                                             ctypes.POINTER(ctypes.c_uint32)]
        lib.mapa_effbw_predict.argtypes = [ctypes.c_int32] * 3 + [ctypes.POINTER(ctypes.c_double)]
        lib.mapa_version.restype = ctypes.c_char_p
        lib.mapa_last_error.restype = ctypes.c_char_p
        lib.mapa_last_error.argtypes = [ctypes.c_void_p]

        def analyze(k, a, b):
            a = np.ascontiguousarray(a, np.int32)
            b = np.ascontiguousarray(b, np.int32)
            aut = ctypes.c_uint64(0)
            back = (ctypes.c_uint32 * max(k, 1))()
            lo = (ctypes.c_uint32 * max(k, 1))()
            rc = lib.mapa_pattern_analyze(k, len(a), a.ctypes.data_as(i32p), b.ctypes.data_as(i32p),
                                          ctypes.byref(aut), back, lo)
            return rc, aut.value

        calls = 0
        for kind, k in itertools.product(("ring", "tree", "clique", "path"), (1, 2, 3, 5, 8, 12, 16, 31, 32)):
            p = W.pattern(kind, k)
            rc, aut = analyze(k, p.a, p.b)
            assert rc == 0, (kind, k, rc)
            calls += 1
        rng = W.Rng(99, 4)
        for trial in range(300):
            k = int(rng.integers(1, 14, 1)[0])
            p = W.random_pattern(rng, k, 0.3, connected=bool(trial % 2))
            rc, aut = analyze(k, p.a, p.b)
            assert rc == 0 and aut >= 1
            calls += 1
        for k, a, b in ((3, [0], [0]), (3, [0], [7]), (3, [-1], [1]), (3, [0, 0], [1, 1]), (0, [], []), (33, [], [])):
            rc, _ = analyze(k, a, b)
            assert rc < 0, (k, a, b)
            calls += 1
        out = ctypes.c_double(0.0)
        for x, y, z in ((0, 0, 0), (2, 1, 0), (3, 1, 0), (63, 63, 63), (64, 0, 0), (-1, 0, 0), (0, 0, 99)):
            lib.mapa_effbw_predict(x, y, z, ctypes.byref(out))
            calls += 1
        assert b"sm_103a" in lib.mapa_version()
        lib.mapa_last_error(None)
        print("child ok", calls)
        """,
        tmp_path,
    )
