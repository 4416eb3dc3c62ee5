"""The row kernels' source hash (build.rows_kernel_sha) leaves comments out,
so that a comment edit keeps a traffic profile valid while any code edit,
string literals included, invalidates it."""
from paper_0906_3611_gb300 import build


def test_comments_are_left_out_and_code_is_kept():
    src = 'int a = 1; // note\n/* block\n comment */ int b = 2;\nasm("x // y");  \n\n'
    got = build._code_only(src)
    assert got == 'int a = 1;\n int b = 2;\nasm("x // y");'
    assert build._code_only("char c = '/'; // x\nchar d = '*';") == "char c = '/';\nchar d = '*';"


def test_a_code_edit_changes_the_hash_and_a_comment_edit_does_not():
    a = "int f() { return 1; } // one\n"
    assert build._code_only(a) == build._code_only("int f() { return 1; } /* uno */\n")
    assert build._code_only(a) != build._code_only("int f() { return 2; } // one\n")


def test_the_hash_is_stable():
    h = build.rows_kernel_sha()
    assert len(h) == 12 and h == build.rows_kernel_sha()
