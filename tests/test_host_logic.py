"""Host-side logic of the benchmark that needs no GPU."""
import bench


def test_kernel_identity_ignores_comments_only():
    a = "int f(int x) {  // add one\n  return x + 1; /* done */ }\n"
    b = "int f(int x) {\n  /* a longer\n     comment */ return x + 1;   }  // new note\n"
    c = "int f(int x) { return x + 2; }"
    assert bench.code_tokens(a) == bench.code_tokens(b) == "int f(int x) { return x + 1; }"
    assert bench.code_tokens(c) != bench.code_tokens(a)


def test_kernel_source_sha_is_stable():
    assert bench.kernel_source_sha() == bench.kernel_source_sha()
    assert len(bench.kernel_source_sha()) == 16
