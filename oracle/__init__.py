"""FP64 CPU oracle of the multiple-block power-spectrum sampler.

TEST INFRASTRUCTURE ONLY.  A plain, slow, obviously correct restatement of the
method of Jasche & Wandelt (arXiv:1306.1821) in FP64 numpy, used to check the
CUDA library element by element.  Only `tests/`, the smoke check in
`__graft_entry__.py` and the `cpu_baseline` / `--impl reference` legs of
`bench.py` may import it.  It shares no code with the CUDA path: it has its own
Philox generator, its own binning and its own samplers; numpy's FFT serves as
the transform step (App. C.1 convention).

Modules (each function cites the section or equation it follows):
    philox  counter-based generator and the uniform / normal transforms
    grid    grid, Fourier convention, half-spectrum weights, k-bins
    model   prior, data model, potential, forces, Hamiltonian
    hmc     momentum draw, leapfrog, HMC move
    draws   Gamma (Marsaglia-Tsang), GIG (ratio of uniforms), normals
    gibbs   P / b / Nbar conditionals, the P-delta jump, the Gibbs scan
    mlp     the mass-preconditioner network (forward, backward, Adam)
    mock    artificial surveys of Sec. 5: field, Poisson and Gaussian counts,
            Schechter selection and mean numbers, bias law, survey response

Pins: every function is checked in tests/test_oracle_*.py against something
other than itself (closed forms, dense linear algebra, finite differences,
quadrature, scipy distributions, an independent Philox implementation).
Parity unpinned: only the sampler's efficiency figures (acceptance ~92%,
correlation length, burn-in length), which the paper reports for its own data.
"""
from . import draws, gibbs, grid, hmc, mlp, mock, model, philox  # noqa: F401
