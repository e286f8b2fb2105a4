"""Shared test helpers: build the library on demand, make solvers from synth workloads."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ensure_built():
    from paper_0707_3405_gb300 import _build
    return _build.build()


def header_functions():
    """Names of every function declared in include/*.h."""
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(lobpcg_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def make_solver(w, **kw):
    """A library Solver for a synth.Workload (projectors in the library's G order)."""
    import paper_0707_3405_gb300 as lg
    return lg.Solver(w.a, w.N, w.ecut, w.kpts, w.vloc(), w.proj_E if w.nproj else None,
                     beta=(lambda mil, k: w.beta(mil, k)) if w.nproj else None, **kw)


def oracle_for(w, solver, k=0):
    """Oracle Hamiltonian in the library's plane-wave order (checked equal as sets)."""
    from oracle import basis, checks, hamiltonian
    mil = solver.gvectors(k).astype(np.int64)
    ref = basis.sphere(w.a, w.N, w.ecut, w.kpts[k])
    perm = checks.map_by_miller(ref, mil)       # ref[perm] == mil
    assert len(perm) == len(ref)
    beta = w.beta(mil, k) if w.nproj else None
    return hamiltonian.Hamiltonian(w.a, w.N, w.kpts[k], mil, w.vloc(), beta, w.proj_E if w.nproj else None)
