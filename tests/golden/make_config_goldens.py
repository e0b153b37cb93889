"""Writes the oracle's expected values for the two large parity workloads, with the harmonic modes
they were computed from (so that a test injects the same ω bits and eigenvector gauge):

  config2_8cubed.npz   seed-0 Morse diamond, 8x8x8 mesh, fixed σ = 0.1 THz, the 8 q points
                       numpy default_rng(0).choice(512, 8) (sorted) x 6 branches, T = 300 K and 700 K
  mesh12_chunks.npz    seed-0 Morse diamond, 12x12x12 mesh (1728 q: more partner points than one
                       chunk of the kernels' q'' lists), fixed σ = 0.02 THz, T = 300 K, 4 modes
  bte_3cubed.npz       seed-0 Morse diamond, 3x3x3 mesh, fixed σ = 0.1 THz, T = 300 K: RTA Γ of
                       every mode and the iterative solution of the linearised BTE (κ of every
                       iterate, the converged F; oracle.Problem.kappa_iterative, tol 1e-12)
  config3_16cubed.npz  seed-1 Morse diamond, 16x16x16 mesh, adaptive σ (scale 1), T = 300 K, the
                       first q point of default_rng(1).choice(4096, 145) (sorted) x 6 branches

Each file holds q, omega [N nb], vel [N nb, 3], evec [N, nb, nb] (complex), T [nT] and, per T,
gamma, wp [nT, 5, n_modes] and counts [nT, 5, n_modes] for the channels 3ph+, 3ph-, 4ph++,
4ph+-, 4ph-- (Algorithms 1 and 4: Γ = C/N^k Σ WP |V|², WP, kept counts).  Only oracle/ and synth/
are called.  Run from the repository root (OpenMP over modes; the 16^3 case takes hours of
one core per mode):

    python tests/golden/make_config_goldens.py config2
    python tests/golden/make_config_goldens.py mesh12
    python tests/golden/make_config_goldens.py bte
    python tests/golden/make_config_goldens.py config3
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = {
    "config2": dict(seed=0, n=8, k=8, sample_seed=0, take=8, sigma=0.1, adaptive=False,
                    temps=(300.0, 700.0), out="config2_8cubed.npz"),
    "mesh12": dict(seed=0, n=12, k=2, sample_seed=12, take=2, sigma=0.02, adaptive=False,
                   temps=(300.0,), out="mesh12_chunks.npz", branches=(1, 5)),
    "config3": dict(seed=1, n=16, k=145, sample_seed=1, take=1, sigma=1.0, adaptive=True,
                    temps=(300.0,), out="config3_16cubed.npz"),
}


def run_bte():
    import oracle
    from synth import morse_system
    P = oracle.Problem(*morse_system(seed=0), (3, 3, 3), T=300.0, sigma=0.1)
    t0 = time.time()
    g, wp, cnt = P.rates()
    k, F, it, ks = P.kappa_iterative(g.sum(0), tol=1e-12, max_iter=200)
    print(f"bte: {it} iterations, {time.time() - t0:.0f} s", flush=True)
    m = P.modes
    np.savez_compressed(os.path.join(HERE, "bte_3cubed.npz"), mesh=np.array((3, 3, 3), np.int32),
                        seed=np.int32(0), sigma=np.float64(0.1), T=np.array([300.0]), omega=m.omega,
                        vel=m.vel, evec=m.evec, gamma=g, kappa=np.array(ks), F=F, iterations=np.int32(it))


def run(name):
    import oracle
    from synth import morse_system, sample_q
    c = CASES[name]
    sysm = morse_system(seed=c["seed"])
    mesh = (c["n"],) * 3
    N = c["n"] ** 3
    q = sample_q(N, c["k"], c["sample_seed"])[:c["take"]]
    nb = sysm[0].nb
    branches = c.get("branches", range(nb))
    modes = np.array([qq * nb + j for qq in q for j in branches], np.int32)
    base = oracle.Problem(*sysm, mesh, T=c["temps"][0], sigma=c["sigma"], sigma_adaptive=c["adaptive"])
    gs, wps, cnts = [], [], []
    for T in c["temps"]:
        P = base.with_T(T)
        t0 = time.time()
        g, wp, cnt = P.rates(modes)
        print(f"{name}: T = {T} K, {modes.size} modes, {cnt.sum()} kept, {time.time() - t0:.0f} s", flush=True)
        gs.append(g)
        wps.append(wp)
        cnts.append(cnt)
    m = base.modes
    np.savez_compressed(os.path.join(HERE, c["out"]), q=q.astype(np.int32), modes=modes,
                        mesh=np.array(mesh, np.int32), seed=np.int32(c["seed"]),
                        sigma=np.float64(c["sigma"]), adaptive=np.int32(c["adaptive"]),
                        T=np.array(c["temps"]), omega=m.omega, vel=m.vel, evec=m.evec,
                        gamma=np.array(gs), wp=np.array(wps), counts=np.array(cnts))


if __name__ == "__main__":
    for name in sys.argv[1:] or ["config2"]:
        run_bte() if name == "bte" else run(name)
