import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


# Offsets whose FP64 oracle value lies within the parity tolerance of a
# threshold, where the FP32 decision may legitimately go either way (the
# reading of bit-exact candidate sets): every candidate-set check records its
# count here, and the session summary reports them.
G13_BAND_COUNTS = []


def record_band_count(what: str, band: int, checked: int) -> None:
    G13_BAND_COUNTS.append((what, int(band), int(checked)))


def pytest_terminal_summary(terminalreporter):
    if not G13_BAND_COUNTS:
        return
    tot = sum(b for _, b, _ in G13_BAND_COUNTS)
    n = sum(c for _, _, c in G13_BAND_COUNTS)
    terminalreporter.write_line("G13 band offsets (decision may go either way): %d of %d offsets checked in %d sets"
                                % (tot, n, len(G13_BAND_COUNTS)))
    for what, b, c in G13_BAND_COUNTS:
        if b:
            terminalreporter.write_line("  %s: %d of %d" % (what, b, c))


def load_golden(name):
    """Parse a hand-derived fixture from tests/golden (format in its README)."""
    path = os.path.join(ROOT, "tests", "golden", name)
    d = {"split": None, "segments": None}
    lines = [ln.strip() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        key, *rest = lines[i].split()
        if key in ("W", "H", "kmax"):
            d[key] = int(rest[0]); i += 1
        elif key in ("sigma", "sigma_used", "rho_max"):
            d[key] = float(rest[0]); i += 1
        elif key == "t":
            d["t"] = [list(map(int, lines[i + 1 + r].split())) for r in range(d["H"])]
            i += 1 + d["H"]
        elif key in ("split", "segments"):
            rows = []
            i += 1
            while i < len(lines) and len(lines[i].split()) == 5 and lines[i].split()[0].lstrip("-").isdigit():
                a = lines[i].split()
                rows.append((int(a[0]), int(a[1]), int(a[2]), int(a[3]), float(a[4])))
                i += 1
            d[key] = rows
        else:
            raise ValueError("bad golden line: " + lines[i])
    return d


GOLDEN = sorted(f for f in os.listdir(os.path.join(ROOT, "tests", "golden")) if f.endswith(".txt") and f != "README.txt")
