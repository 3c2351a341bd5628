"""Planted mistakes: a copy of oracle.c with one textual change, built on the
CPU into a temporary directory, so that a test can show that its pin fails
when the oracle is wrong in a plausible way.  The oracle under test is never
modified; the copy is loaded through oracle.use_library for the duration of
the check."""
from __future__ import annotations

import contextlib
import shutil
import subprocess
import tempfile
from pathlib import Path

ORACLE_DIR = Path(__file__).resolve().parent.parent / "oracle"


def build_planted(replacements: list[tuple[str, str]], workdir: Path | None = None) -> Path:
    """Builds liboracle.so from oracle.c with each (old, new) replacement made
    exactly once; returns the library path."""
    src = (ORACLE_DIR / "oracle.c").read_text()
    for old, new in replacements:
        n = src.count(old)
        if n != 1:
            raise ValueError(f"planted mistake: {old!r} occurs {n} times in oracle.c")
        src = src.replace(old, new)
    d = Path(workdir or tempfile.mkdtemp(prefix="planted_oracle_"))
    (d / "oracle.c").write_text(src)
    shutil.copy(ORACLE_DIR / "oracle.h", d / "oracle.h")
    lib = d / "liboracle.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-fno-fast-math",
                    "-ffp-contract=off", str(d / "oracle.c"), "-o", str(lib), "-lm"], check=True)
    return lib


@contextlib.contextmanager
def planted(replacements: list[tuple[str, str]]):
    """Context in which the oracle module runs the planted copy."""
    from oracle import oracle
    d = Path(tempfile.mkdtemp(prefix="planted_oracle_"))
    try:
        lib = build_planted(replacements, d)
        with oracle.use_library(lib):
            yield oracle
    finally:
        shutil.rmtree(d, ignore_errors=True)
