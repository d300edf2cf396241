#!/usr/bin/env python3
"""Writes the stored expected values under tests/golden/ by calling only the
CPU oracle (oracle/) on inputs from the seeded generators (graphgen/).  No
value here comes from the CUDA library.

  python tests/golden/make_golden.py rmat22_tr_eo --p 0.2 0.5 0.8
      R-MAT scale 22, edge factor 16, seed 1 (the benchmark's edge-once
      config); for each p, the oracle's Edge-Once p-1-TR output (Sec. 4.3;
      Sec. 6, Edge-Once p-1-TR) with compression seed 1: its arc count and
      CSR digest.  About half an hour of one core per p and up to 34 GB of
      host memory (p = 0.8: 1.7e9 selected triangles, 16 bytes each).

  python tests/golden/make_golden.py chung_lu26_mst [--device cuda]
      Chung-Lu, 2^26 vertices, exponent 2.1, mean degree 32, weights
      k * 2^-24 (seed 1): the oracle's Kruskal MST weight in units of 2^-24
      and its component count.  The generator may run on a GPU (input
      generation only); the oracle runs on the host.

Entries are merged into the golden file by key, so runs for different p may
go in separate processes.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402
from tests.digest import csr_digest, read_golden  # noqa: E402

HEADERS = {
    "rmat22_tr_eo": (
        "# Edge-Once p-1-TR (Sec. 4.3; Sec. 6, Edge-Once p-1-TR) of R-MAT scale 22, edge factor 16,\n"
        "# (a,b,c) = (.57,.19,.19), generator seed 1, compression seed 1, by the CPU oracle.\n"
        "# Written by tests/golden/make_golden.py rmat22_tr_eo (calls only oracle/ and graphgen/).\n"
        "# graph <n> <nnz> <sha256 of the input CSR>\n"
        "# p<p> <arcs of H> <sha256 of H's CSR>  (digest: tests/digest.py)\n"),
    "chung_lu26_mst": (
        "# Chung-Lu 2^26 vertices, exponent 2.1, mean degree 32, weights k*2^-24 (seed 1), by the CPU oracle:\n"
        "# Kruskal MST weight in units of 2^-24 and the component count (Sec. 6 \"Others\": max-weight TR\n"
        "# keeps both).  Written by tests/golden/make_golden.py chung_lu26_mst (calls only oracle/ and graphgen/).\n"
        "# graph <n> <nnz> <sha256 of the input CSR with weights>\n"
        "# mst_units <units>\n"
        "# cc <components>\n"),
}


def _merge(name: str, entries: dict):
    path = os.path.join(HERE, name + ".txt")
    old = read_golden(path) if os.path.exists(path) else {}
    old.update({k: [str(x) for x in v] for k, v in entries.items()})
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        f.write(HEADERS[name])
        for k in sorted(old, key=lambda k: (k != "graph", k)):
            f.write(" ".join([k, *old[k]]) + "\n")
    os.replace(tmp, path)


def rmat22_tr_eo(ps, device):
    t0 = time.time()
    g = gg.rmat(22, 16, seed=1, device=device).to("cpu")
    off, col, _ = g.numpy()
    _merge("rmat22_tr_eo", {"graph": [g.n, g.nnz, csr_digest(off, col)]})
    print(f"generated n={g.n} nnz={g.nnz} in {time.time() - t0:.0f} s", flush=True)
    for p in ps:
        t0 = time.time()
        o_off, o_col, _ = oracle.compress(g, "tr_eo", p, 1)
        _merge("rmat22_tr_eo", {f"p{p}": [o_col.size, csr_digest(o_off, o_col)]})
        print(f"p={p}: {o_col.size} arcs kept, {time.time() - t0:.0f} s", flush=True)


def chung_lu26_mst(device):
    t0 = time.time()
    g = gg.attach_weights(gg.chung_lu(26, 2.1, 32.0, seed=1, device=device), seed=1).to("cpu")
    off, col, w = g.numpy()
    _merge("chung_lu26_mst", {"graph": [g.n, g.nnz, csr_digest(off, col, w)]})
    print(f"generated n={g.n} nnz={g.nnz} in {time.time() - t0:.0f} s", flush=True)
    t0 = time.time()
    units = oracle.mst_weight_units(g)
    cc = oracle.cc_count(g)
    _merge("chung_lu26_mst", {"mst_units": [units], "cc": [cc]})
    print(f"mst_units={units} cc={cc} in {time.time() - t0:.0f} s", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=sorted(HEADERS))
    ap.add_argument("--p", type=float, nargs="+", default=[0.2, 0.5, 0.8])
    ap.add_argument("--device", default="cpu", help="where graphgen builds the input (cpu or cuda)")
    a = ap.parse_args()
    oracle.build()
    if a.what == "rmat22_tr_eo":
        rmat22_tr_eo(a.p, a.device)
    else:
        chung_lu26_mst(a.device)


if __name__ == "__main__":
    main()
