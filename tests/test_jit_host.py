"""Runtime specialisation (NVRTC) on the host: compiling the element kernel
for user expressions needs no GPU, so the compile step, its cache and its
input checks are tested here; the compiled kernels run in test_gpu_jit.py."""
import pytest

from paper_1802_03433_gb300 import build_lib

K_EXPR = "1 + 0.5*sin(3*x)*cos(2*y) + z*z"
F_EXPR = "p0*sinpi_fp64(x)*sinpi_fp64(y)*sinpi_fp64(z)"


@pytest.fixture(scope="module")
def fea():
    build_lib.build()
    from paper_1802_03433_gb300 import fea as f
    return f


@pytest.mark.parametrize("order,kind,npts,prec", [(1, 0, 1, 0), (1, 0, 4, 1), (2, 1, 11, 0), (2, 1, 4, 1)])
def test_compiles_to_a_cubin(fea, order, kind, npts, prec):
    j = fea.fea_jit_compile(fea.make_form(kind, order, 1.0), fea.make_quadrature(npts, prec), K_EXPR, F_EXPR)
    ms, nbytes, hit = fea.fea_jit_info(j)
    src = fea.fea_jit_source(j)
    assert nbytes > 1000 and ms > 0
    assert K_EXPR in src and F_EXPR in src
    assert f"elem_user_body<{order}, {'true' if kind == 1 else 'false'}, {npts}, " \
           f"{'double' if prec == 0 else 'float'}, fea::UserSpec>" in src
    fea.fea_jit_destroy(j)


def test_same_specialisation_is_cached(fea):
    form, q = fea.make_form(0, 1), fea.make_quadrature(4)
    a = fea.fea_jit_compile(form, q, "2 + x*y - 0.25*z", None)
    b = fea.fea_jit_compile(form, q, "2 + x*y - 0.25*z", None)
    c = fea.fea_jit_compile(form, q, "2 + x*y - 0.5*z", None)
    assert fea.fea_jit_info(b)[2] and not fea.fea_jit_info(c)[2]
    assert fea.fea_jit_info(a)[1] == fea.fea_jit_info(b)[1]
    for h in (a, b, c):
        fea.fea_jit_destroy(h)


@pytest.mark.parametrize("kind,prec", [(1, 0), (0, 0), (1, 1), (0, 1)])
def test_no_expressions_gives_the_constant_coefficient_kernel(fea, kind, prec):
    """P2 without k(x): the closed-form entries of the precompiled kernels'
    FMA chains, FP64 and FP32, with and without mass."""
    j = fea.fea_jit_compile(fea.make_form(kind, 2, 1.0 if kind else 0.0), fea.make_quadrature(11, prec), None, None)
    src = fea.fea_jit_source(j)
    assert "HAS_K = false" in src and "HAS_F = false" in src
    assert f"elem_user_body<2, {'true' if kind else 'false'}, 11, {'double' if prec == 0 else 'float'}," in src
    assert fea.fea_jit_info(j)[1] > 1000
    fea.fea_jit_destroy(j)


@pytest.mark.parametrize("bad,msg", [
    ("x; int a", "';' is not allowed"), ("x) { return 0", "not allowed"), ("#define X", "not allowed"),
    ("(x + 1", "unbalanced"), ("x) + (y", "unbalanced"), ("x // c", "comments"), ("x /* c */", "comments"),
    ("\"s\"", "not allowed"), ("", "empty"), ("x" * 5000, "longer"), ("undefined_fn(x)", "NVRTC could not compile")])
def test_bad_expressions_are_rejected(fea, bad, msg):
    with pytest.raises(fea.FeaError) as e:
        fea.fea_jit_compile(fea.make_form(0, 1), fea.make_quadrature(4), bad, None)
    assert msg in str(e.value)


@pytest.mark.parametrize("form,quad,msg", [
    ((2, 1), (4, 0), "scalar forms"), ((0, 3), (4, 0), "order"), ((0, 1), (5, 0), "npts"), ((0, 1), (4, 7), "prec")])
def test_bad_specialisations_are_rejected(fea, form, quad, msg):
    with pytest.raises(fea.FeaError) as e:
        fea.fea_jit_compile(fea.make_form(*form), fea.make_quadrature(*quad), "1", None)
    assert msg in str(e.value)
