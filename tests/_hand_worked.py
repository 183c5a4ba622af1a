"""Page images worked by hand from the storage-format definition.

Closed forms: each entry gives the input column, the derivation done by
hand, and the expected bytes of the encoded page.  Nothing here was produced
by a program.  Format: a 16-byte page header {'D','P','F',codec; nrows;
payload offset; string-region offset}, then the mini block headers, zero
padding to 16 bytes, the packed payload (value j of a mini block at bit
j*bw, LSB first, in little-endian 32-bit words), and for strings the raw
bytes (Sec. 3.4.1 fixed-length layout, Sec. 3.4.2 variable-length layout,
Sec. 4.1 GPU-FOR, Sec. 4.2 page metadata).
"""


def _h(*parts):
    return "".join(parts)


HAND_WORKED = [
    dict(name="for_bw4_nibbles", codec="for", page_rows=128,
         values=[1000 + (j % 16) for j in range(128)],
         cite="Sec. 3.4.1 mini blocks (FOR base, bit width, byte offset); Sec. 4.1 GPU-FOR for INT32",
         derivation="base=1000, span 15 -> bw=4; p_j=j%16, 8 per word: even words "
                    "0x76543210, odd words 0xfedcba98; header {1000, (0<<8)|4}; payload "
                    "at byte 32 = 16-byte page header + 8-byte header, rounded to 16",
         page_hex=_h("44504601", "80000000", "20000000", "00000000", "e8030000", "04000000",
                     "0000000000000000", "1032547698badcfe" * 8),
         page_off=[0, 96], row_prefix=[128]),
    dict(name="for_constant_bw0", codec="for", page_rows=128, values=[-7] * 5,
         cite="Sec. 3.4.1; a constant mini block needs no packed words",
         derivation="max==min -> bw=0; base=-7=0xfffffff9; nrows=5",
         page_hex=_h("44504601", "05000000", "20000000", "00000000", "f9ffffff", "00000000",
                     "0000000000000000"),
         page_off=[0, 32], row_prefix=[5]),
    dict(name="for_bw1_alternating", codec="for", page_rows=128,
         values=[5 + (j % 2) for j in range(128)],
         cite="Sec. 3.4.1",
         derivation="base=5, bw=1, bit j = j%2 -> each of the 4 words is 0xaaaaaaaa",
         page_hex=_h("44504601", "80000000", "20000000", "00000000", "05000000", "01000000",
                     "0000000000000000", "aaaaaaaa" * 4),
         page_off=[0, 48], row_prefix=[128]),
    dict(name="delta_arithmetic", codec="delta", page_rows=128,
         values=[100 + 3 * j for j in range(128)],
         cite="delta-coded keys over Sec. 3.4.1 mini blocks (sorted loads, Sec. 4.2)",
         derivation="d_0=0, d_j=3 -> dmin=0, span 3 -> bw=2; p_0=0, p_j=3 -> "
                    "word0=0xfffffffc, words 1..7=0xffffffff; header {first=100, dmin=0, 2, 0}",
         page_hex=_h("44504602", "80000000", "20000000", "00000000", "64000000", "00000000",
                     "02000000", "00000000", "fcffffff", "ffffffff" * 7),
         page_off=[0, 64], row_prefix=[128]),
    dict(name="delta_descending_ragged", codec="delta", page_rows=128, values=[10, 7, 4],
         cite="delta-coded integers; ragged last mini block",
         derivation="d=(0,-3,-3) -> dmin=-3, span 3 -> bw=2; p=(3,0,0), padding p=0 -> "
                    "word0=3; header {10, 0xfffffffd, 2, 0}",
         page_hex=_h("44504602", "03000000", "20000000", "00000000", "0a000000", "fdffffff",
                     "02000000", "00000000", "03000000", "00000000" * 7),
         page_off=[0, 64], row_prefix=[3]),
    dict(name="dict_codes", codec="dict", page_rows=128, values=[30, 10, 20, 10],
         cite="Sec. 3.4.1 (short CHAR reinterpreted as integers, then GPU-FOR): codes are FOR-packed",
         derivation="dictionary (10,20,30); codes (2,0,1,0) -> base 0, bw 2 -> "
                    "word0 = 2 | 0<<2 | 1<<4 | 0<<6 = 0x12",
         dict=[10, 20, 30],
         page_hex=_h("44504603", "04000000", "20000000", "00000000", "00000000", "02000000",
                     "0000000000000000", "12000000", "00000000" * 7),
         page_off=[0, 64], row_prefix=[4]),
    dict(name="str_three_rows", codec="str", page_rows=128, strings=[b"ab", b"", b"xyz"],
         cite="Sec. 3.4.2 variable-length page, offsets stored as FOR-packed lengths",
         derivation="lengths (2,0,3): base 0, bw 2 -> word0 = 2 | 0<<2 | 3<<4 = 0x32; header "
                    "{0, 2}, then start 0; payload at align16(16+12)=32 (8 words); bytes at "
                    "align16(32+32)=64: 'abxyz', page padded to 80",
         page_hex=_h("44504604", "03000000", "20000000", "40000000", "00000000", "02000000",
                     "00000000", "00000000", "32000000", "00000000" * 7, "616278797a",
                     "00" * 11),
         page_off=[0, 80], row_prefix=[3]),
    dict(name="for_two_pages_ragged", codec="for", page_rows=128, values=list(range(200)),
         cite="Sec. 3.4.2 RID index (cumulative rows up to and including page i); Sec. 4.2 page offsets",
         derivation="page 0: rows 0..127, bw 7 -> 28 words -> 32+112=144 bytes; page 1: rows "
                    "128..199, base 128, span 71 -> bw 7 -> 144 bytes; page-0 word0 = "
                    "0|1<<7|2<<14|3<<21|(4&15)<<28 = 0x40608080, word1 = "
                    "4>>4|5<<3|6<<10|7<<17|8<<24|(9&1)<<31 = 0x880e1828",
         page0_payload_prefix_hex="80806040" "28180e88",
         page_off=[0, 144, 288], row_prefix=[128, 200]),
]
