"""binary64 mode: forward and hand-written backward through the exact path,
against the oracle (stage by stage, bit for bit), the exact product and the
exact central finite difference of L(A, B) = <G, A B> (each <= 1 ulp)."""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import ozaki2_oracle as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def ag():
    from paper_2609_27831_gb300 import build
    build.build()
    from paper_2609_27831_gb300 import autograd
    return autograd


def _ulps(x: float, ref: float) -> Fraction:
    return o.ulp_distance(Fraction(x), Fraction(ref), 53) if ref else Fraction(abs(x))


def _fd_grad_A(X, Y, G, i, k):
    """Exact central difference of <G, A B> in A_ik (bilinear: exact for any h)."""
    h = Fraction(1, 3)
    def loss(delta):
        tot = Fraction(0)
        for j in range(Y.shape[1]):
            s = Fraction(0)
            for kk in range(X.shape[1]):
                a = Fraction(float(X[i, kk])) + (delta if kk == k else 0)
                s += a * Fraction(float(Y[kk, j]))
            tot += Fraction(float(G[i, j])) * s
        return tot
    return float((loss(h) - loss(-h)) / (2 * h))


def _fd_grad_B(X, Y, G, k, j):
    """Exact central difference of <G, A B> in B_kj."""
    h = Fraction(1, 5)
    def loss(delta):
        tot = Fraction(0)
        for i in range(X.shape[0]):
            s = Fraction(0)
            for kk in range(X.shape[1]):
                b = Fraction(float(Y[kk, j])) + (delta if kk == k else 0)
                s += Fraction(float(X[i, kk])) * b
            tot += Fraction(float(G[i, j])) * s
        return tot
    return float((loss(h) - loss(-h)) / (2 * h))


@pytest.mark.parametrize("M,N,K", [(24, 16, 40), (130, 70, 300), (64, 300, 33)])
def test_forward_backward_against_oracle(ag, M, N, K):
    rng = np.random.Generator(np.random.PCG64(3000 + M))
    X = synth.fp64_matrix(rng, M, K)
    Y = synth.fp64_matrix(rng, K, N)
    G = synth.fp64_normal(rng, M, N)
    xa = torch.tensor(X, device="cuda", requires_grad=True)
    ya = torch.tensor(Y, device="cuda", requires_grad=True)
    out = ag.ozaki_matmul(xa, ya)
    out.backward(torch.tensor(G, device="cuda"))
    torch.cuda.synchronize()
    C_, dA, dB = out.detach().cpu().numpy(), xa.grad.cpu().numpy(), ya.grad.cpu().numpy()
    par = o.dgemm_params(M, N, K)
    e, f = o.f64_exponents(X, 1), o.f64_exponents(Y, 0)
    rnd = np.random.Generator(np.random.PCG64(9))
    for _ in range(12):
        i, j, k = int(rnd.integers(M)), int(rnd.integers(N)), int(rnd.integers(K))
        assert C_[i, j] == o.dgemm_fwd_entry(X, Y, i, j, par, e, f)
        assert dA[i, k] == o.dgemm_dA_entry(Y, G, i, k, par, f)
        assert dB[k, j] == o.dgemm_dB_entry(X, G, k, j, par, e)
        assert _ulps(C_[i, j], o.exact_dot_double(X[i, :], Y[:, j])) <= 1
        assert _ulps(dA[i, k], o.exact_dot_double(G[i, :], Y[k, :])) <= 1
        assert _ulps(dB[k, j], o.exact_dot_double(X[:, k], G[:, j])) <= 1
    i, k = 1, 2
    assert _ulps(dA[i, k], _fd_grad_A(X, Y, G, i, k)) <= 1
    k, j = 3, 1
    assert _ulps(dB[k, j], _fd_grad_B(X, Y, G, k, j)) <= 1


def test_backward_only_one_side(ag):
    rng = np.random.Generator(np.random.PCG64(3100))
    X = synth.fp64_matrix(rng, 20, 30)
    Y = synth.fp64_matrix(rng, 30, 10)
    xa = torch.tensor(X, device="cuda", requires_grad=True)
    ya = torch.tensor(Y, device="cuda")
    out = ag.ozaki_matmul(xa, ya)
    out.sum().backward()
    torch.cuda.synchronize()
    G = np.ones((20, 10))
    par = o.dgemm_params(20, 10, 30)
    assert xa.grad[3, 4].item() == o.dgemm_dA_entry(Y, G, 3, 4, par)
