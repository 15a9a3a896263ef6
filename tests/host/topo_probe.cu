// Test probe (host code only, no GPU needed): prints the library's closed-form
// level-order topology maps and float sort keys so that a CPU test can compare
// them with an independent enumeration.
//
// stdin lines:  "t <n> <t>"  ->  "<level> <inorder(t)> <node_at(t)> <leftmost(t)> <rightmost(t)>"
//               "k <bits>"   ->  "<float_key(bits as float)>"
#include <cstdio>
#include <cstring>

#include "../../paper_2210_12859_gb300/csrc/kdt_internal.cuh"

int main()
{
    char op[4];
    while (scanf("%3s", op) == 1) {
        if (op[0] == 't') {
            long long n, t;
            if (scanf("%lld %lld", &n, &t) != 2)
                return 2;
            kdt::Topo T(n);
            printf("%d %lld %lld %lld %lld\n", kdt::Topo::level(t), (long long)T.inorder(t), (long long)T.node_at(t),
                   (long long)T.leftmost(t), (long long)T.rightmost(t));
        } else if (op[0] == 'k') {
            unsigned bits;
            if (scanf("%x", &bits) != 1)
                return 2;
            float x;
            memcpy(&x, &bits, 4);
            printf("%u\n", kdt::float_key(x));
        } else {
            return 2;
        }
    }
    return 0;
}
