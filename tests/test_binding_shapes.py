"""The binding rejects a field of the wrong shape before any pointer reaches
the library: the C side reads and writes exactly 3*N (vector) or N (scalar)
floats through each pointer, so an undersized or misshapen tensor must never
get that far.  CPU only: the checks run before the library is touched."""
import pytest

torch = pytest.importorskip("torch")

from paper_2008_12820_gb300 import claire as C


def fake_registration(shape=(8, 8, 8)):
    """A Registration whose context was never created (no GPU needed): any
    call that got past the argument checks would fail on the NULL handle."""
    reg = object.__new__(C.Registration)
    reg._h = None
    reg.shape = tuple(shape)
    return reg


def test_vector_and_scalar_shapes_are_checked_first():
    reg = fake_registration()
    bad_vec = [torch.zeros(2, 8, 8, 8), torch.zeros(3, 8, 8, 7), torch.zeros(3 * 8 * 8 * 8), torch.zeros(8, 8, 8)]
    for t in bad_vec:
        for call in (lambda t: reg.gradient(t), lambda t: reg.linearize(t), lambda t: reg.precond(t),
                     lambda t: reg.apply_A(t), lambda t: reg.objective(t), lambda t: reg.div(t),
                     lambda t: reg.hess_matvec(None, t), lambda t: reg.solve(t)):
            with pytest.raises(ValueError, match="shape"):
                call(t)
    for t in (torch.zeros(8, 8, 9), torch.zeros(3, 8, 8, 8), torch.zeros(512)):
        with pytest.raises(ValueError, match="shape"):
            reg.set_images(t, t)
        with pytest.raises(ValueError, match="shape"):
            reg.grad(t)
    # a host tensor of the right shape is refused too (device memory only)
    with pytest.raises(ValueError, match="CUDA"):
        reg.precond(torch.zeros(3, 8, 8, 8))


def test_host_solve_shapes_are_checked():
    reg = fake_registration()
    m = torch.zeros(8, 8, 8)
    with pytest.raises(ValueError, match="shape"):
        reg.solve_host(m, m, torch.zeros(3, 8, 8, 4))
    with pytest.raises(ValueError, match="shape"):
        reg.solve_host(torch.zeros(8, 8, 4), m, torch.zeros(3, 8, 8, 8))


def test_precond_noalloc_shapes_are_checked():
    for r, s in ((torch.zeros(2, 8, 8, 8), torch.zeros(2, 8, 8, 8)),
                 (torch.zeros(8, 8, 8), torch.zeros(8, 8, 8)),
                 (torch.zeros(3, 8, 8, 8), torch.zeros(3, 8, 8, 4))):
        with pytest.raises(ValueError):
            C.precond_noalloc(r, s, 1e-2, 1.0)
