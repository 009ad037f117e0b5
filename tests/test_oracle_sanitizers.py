"""The FP64 oracle runs its pins clean under AddressSanitizer and UBSan.

A memory error in the oracle would silently corrupt every parity verdict, so
its C source is compiled with -fsanitize=address,undefined into a temporary
directory and the pins of ``test_oracle_pins.py`` run against that build in a
child process (the sanitizer runtimes preloaded, since Python itself is not
instrumented).  A control plants a one-past-the-end read in a copy and checks
that the same harness reports it.  CPU only; skipped where gcc has no
sanitizer runtimes.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dscreen_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")
FLAGS = ["-O1", "-g", "-std=c99", "-fPIC", "-shared", "-fsanitize=address,undefined",
         "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer"]

_CHILD = (
    "import sys\n"
    "sys.path.insert(0, {root!r})\n"
    "import oracle\n"
    "oracle._SRC, oracle._BUILD, oracle._LIB = {src!r}, {bdir!r}, {lib!r}\n"
    "import pytest\n"
    "sys.exit(pytest.main([{pins!r}, '-x', '-q', '-s', '-p', 'no:cacheprovider', '-k', {sel!r}]))\n"
)


def _runtimes():
    libs = []
    for name in ("libasan.so", "libubsan.so"):
        p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
        if not os.path.isabs(p) or not os.path.exists(p):
            pytest.skip(f"gcc has no {name}")
        libs.append(p)
    return " ".join(libs)


def _run(text, bdir, sel):
    os.makedirs(bdir)
    src = os.path.join(bdir, "dscreen_oracle.c")
    lib = os.path.join(bdir, "liboracle.so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", *FLAGS, "-o", lib, src, "-lm"])
    env = dict(os.environ, LD_PRELOAD=_runtimes(), ASAN_OPTIONS="detect_leaks=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    code = _CHILD.format(root=ROOT, src=src, bdir=bdir, lib=lib, pins=PINS, sel=sel)
    p = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    return p.returncode, p.stdout + p.stderr


def _reported(out):
    return "runtime error" in out or "AddressSanitizer" in out


def test_pins_run_clean_under_sanitizers(tmp_path):
    with open(SRC) as f:
        base = f.read()
    rc, out = _run(base, str(tmp_path / "clean"), "not dome_max_matches_numeric_maximum")
    assert rc == 0 and not _reported(out), out[-3000:]


def test_sanitized_build_reports_a_planted_overrun(tmp_path):
    with open(SRC) as f:
        base = f.read()
    old = "for (int64_t i = 0; i < K; i++) x_out[i] = x[i];"
    assert base.count(old) == 1
    rc, out = _run(base.replace(old, "for (int64_t i = 0; i <= K; i++) x_out[i % K] = x[i];"),
                   str(tmp_path / "planted"), "lambda_max")
    assert rc != 0 and _reported(out), out[-3000:]
